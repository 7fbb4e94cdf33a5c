// Mixed-precision step: the propagation, Gram and U R^-1 products run on the
// tensor cores as split-fp16 GEMMs (gemm_tc.cu); occupations, the homodyne
// weight and the projective updates on the CUDA cores in float / double; the
// Cholesky factor and its inverse in float64.
//
// State layout: trajectory b holds V_b (2L x N float, column-major): column k
// is [Re U_{:,k}; Im U_{:,k}].  Read as an L x 2N column-major matrix, V_b is
// U~ = [Re u_0, Im u_0, Re u_1, ...].
//   propagation  V' = [[Re P, -Im P], [Im P, Re P]] V          (A: 2L x 2L, B: V)
//   Gram         Re G = V^T V,  Im G_kl = sum_s V_sk V_{(s+L) mod 2L, l} (-1)^{s >= L}
//   U R^-1       U~' = U~ T~,  T~ the real 2N x 2N embedding of T = R^-1
#include <algorithm>
#include <vector>

#include "fm_testing.h"
#include "gemm_tc.h"
#include "mixed.h"

namespace fm {

namespace {

// tile width of the propagation and Gram products, raster group height (fm.h, FM_TILE_*).
// Defaults (measured): up to N = 8192, 128-wide tiles (two TMEM accumulator sets, so a
// tile's epilogue overlaps the next tile's products: the Gram at L = 16384 takes 63 ms
// instead of 79 ms per pair of passes, the propagation is unchanged); beyond, 256-wide
// tiles, whose operand panels are read half as often (the 160 x 160 torus Gram: 614 ms
// instead of 904 ms); raster groups of 8 row tiles.
int pick_bn(int N, int tile_config) {
  const int c = tile_config & 3;
  if (c == 1) return 128;
  if (c == 2) return 256;
  return (N > 8192 && N % 256 == 0) ? 256 : 128;
}
int pick_gm(int tile_config) {
  const int g = (tile_config >> 2) & 7;
  return g ? (1 << (g + 1)) : 8;
}

// Second-pass guard, in device memory: per trajectory b the largest |diag E| and
// off-diagonal |E| (float bits, E = G - 1 of the second pass's Gram) in e2[2b], e2[2b+1];
// the same for the conditional extra pass in e3; the extra-pass flag; counters (second
// passes checked, extra passes run); the running maxima since the last query (e2 diag,
// e2 off-diagonal, e3 diag, e3 off-diagonal, float bits).
struct GuardPtrs {
  unsigned *e2, *e3;
  int* flag;
  unsigned long long* counters;
  unsigned* seen;
};
size_t guard_bytes(int B) { return (size_t)16 * B + 64; }
GuardPtrs guard_ptrs(void* base, int B) {
  GuardPtrs g;
  char* p = (char*)base;
  g.counters = (unsigned long long*)p;          // [0] checks, [1] extra passes
  g.seen = (unsigned*)(p + 16);                 // [4]
  g.flag = (int*)(p + 32);
  g.e2 = (unsigned*)(p + 64);
  g.e3 = g.e2 + 2 * B;
  return g;
}

struct Scratch {
  size_t total = 0;
  size_t tiles_prop, tiles_gram, tiles_trmm, tiles_trmm2, urm_h, urm_l;
  // block projective update (pm_block.cu), projective states that use it only
  size_t pb_list, pb_ulist, pb_count, pb_pos, pb_wt_h, pb_wt_l, pb_dp, pb_dph, pb_dpl, pb_ap, pb_ath, pb_atl;
  size_t pb_tth, pb_ttl, pb_xth, pb_xtl, pb_mats, pb_vecs, pb_ev, pb_wc, pb_x;
  int pb_kc = 0;
  size_t ca_h, ca_l, cb_h, cb_l, xs;       // complex tensor GEMM helper (Cholesky recursion)
  size_t gf, rf, tf, dinvf, xf, diag;     // complex64 Gram / factor / inverse, FP64 Gram diagonal
  size_t guard;                           // second-pass guard (ReorthGuard layout)
  size_t take(size_t b) { size_t o = total; total += (b + 255) & ~(size_t)255; return o; }
};

// mixed-precision projective steps run as blocks (pm_block.cu); the per-event
// paths remain for steps that select more sites than the block holds
bool uses_pm_block(int protocol, int L, int B) {
  (void)L;
  (void)B;
  return protocol == FM_PROJECTIVE;
}

Scratch scratch_plan(int Lx, int Ly, int B, int protocol) {
  Scratch s;
  const int64_t L = (int64_t)Lx * Ly, N = L / 2;
  const int BN = 128;                              // the longer tile lists of either width
  const int64_t n_prop = (2 * L / tc::BM) * (B * N / BN);
  const int64_t n_gram = (int64_t)B * 2 * (N / tc::BM) * (N / BN);
  const int64_t n_trmm = (int64_t)B * (L / tc::BM) * (2 * N / 128);
  s.tiles_prop = s.take(n_prop * 16);
  s.tiles_gram = s.take(n_gram * 16);
  s.tiles_trmm = s.take(n_trmm * 16);
  s.tiles_trmm2 = s.take(n_trmm / 2 * 16);        // second pass: 256-wide tiles
  s.urm_h = s.take((int64_t)B * L * 2 * N * 2);
  s.urm_l = s.take((int64_t)B * L * 2 * N * 2);
  const int64_t md = N / 2 + 128;                  // largest block the recursion multiplies
  s.ca_h = s.take((int64_t)B * 4 * md * md * 2);
  s.ca_l = s.take((int64_t)B * 4 * md * md * 2);
  s.cb_h = s.take((int64_t)B * 2 * md * md * 2);
  s.cb_l = s.take((int64_t)B * 2 * md * md * 2);
  s.xs = s.take((int64_t)B * md * md * 8);
  s.gf = s.take((int64_t)B * N * N * 8);
  s.rf = s.take((int64_t)B * N * N * 8);
  s.tf = s.take((int64_t)B * N * N * 8);
  s.dinvf = s.take((int64_t)B * ((N + 31) / 32) * 32 * 32 * 8);
  s.xf = s.take((int64_t)B * N * 32 * 8);
  s.diag = s.take((int64_t)B * N * 8);
  s.guard = s.take(guard_bytes(B));
  if (uses_pm_block(protocol, (int)L, B)) {
    const int64_t Kc = pmb_capacity((int)L);
    s.pb_kc = (int)Kc;
    s.pb_list = s.take(B * L * 4);
    s.pb_ulist = s.take(B * L * 8);
    s.pb_count = s.take(B * 4);
    s.pb_pos = s.take(B * L * 4);
    // every operand for all trajectories, so that each product is one launch
    s.pb_wt_h = s.take(B * 2 * Kc * 2 * N * 2);
    s.pb_wt_l = s.take(B * 2 * Kc * 2 * N * 2);
    s.pb_dp = s.take(B * L * 2 * Kc * 4);
    s.pb_dph = s.take(B * L * 2 * Kc * 2);
    s.pb_dpl = s.take(B * L * 2 * Kc * 2);
    s.pb_ap = s.take(B * L * 2 * Kc * 4);
    s.pb_ath = s.take(B * 2 * L * 2 * Kc * 2);
    s.pb_atl = s.take(B * 2 * L * 2 * Kc * 2);
    s.pb_tth = s.take(B * 2 * Kc * 2 * Kc * 2);
    s.pb_ttl = s.take(B * 2 * Kc * 2 * Kc * 2);
    s.pb_xth = s.take(B * N * 2 * Kc * 2);
    s.pb_xtl = s.take(B * N * 2 * Kc * 2);
    s.pb_mats = s.take(7 * B * Kc * Kc * 8);
    s.pb_vecs = s.take(4 * B * Kc * 8);
    s.pb_ev = s.take(B * (int64_t)sizeof(PmbEvent));
    s.pb_wc = s.take(B * Kc * N * 8);
    s.pb_x = s.take(B * Kc * N * 8);
  }
  return s;
}

// ------------------------------------------------------------------ kernels

FM_DEVFN void split16_f(float v, __half& h, __half& l) {
  h = __float2half_rn(v);
  l = __float2half_rn((v - __half2float(h)) * 2048.0f);
}

// K-major planes of the real embedding of an upper-triangular N x N complex
// matrix Z (rows c, K index j, 2N x 2N per trajectory):
//   Z~[2l+s, 2n+s'] = Re Z_ln (s = s'), Im Z_ln (s=0, s'=1), -Im Z_ln (s=1, s'=0).
// mode 0: Z = T - 1 (T = R^-1 from the Cholesky recursion);
// mode 1: Z = -F, F = strict upper part of G plus half of (diag G - 1) (the
//         diagonal taken from the float64 Gram diagonal): the first-order
//         inverse factor of G = 1 + E, (1 + F)^dag (1 + F) = G + O(E^2).
// One block per row (b, c) of Z~ (2N halves), eight K positions per thread and
// pass, written as 16-byte stores of each plane.
__global__ void __launch_bounds__(256) build_ttilde_kernel(const c32* __restrict__ Z, const double* __restrict__ diag,
                                                           int mode, int N, __half* Th, __half* Tl, const int* cond) {
  if (cond && *cond == 0) return;
  const int N2 = 2 * N;
  const int64_t row = blockIdx.x;
  const int64_t b = row / N2;
  const int c = (int)(row - b * N2);
  const int n = c >> 1, sp = c & 1;
  const c32* Zc = Z + b * (int64_t)N * N + (int64_t)n * N;   // column n
  __half* th = Th + row * N2;
  __half* tl = Tl + row * N2;
  for (int j0 = threadIdx.x * 8; j0 < N2; j0 += blockDim.x * 8) {
    __align__(16) __half hh[8];
    __align__(16) __half ll[8];
    const int l0 = j0 >> 1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int l = l0 + q;
      float re = 0.0f, im = 0.0f;
      if (l <= n) {
        c32 z = Zc[l];
        if (mode == 0) {
          if (l == n) z.re -= 1.0f;
        } else if (l == n) {
          z.re = (float)(-(diag[b * N + n] - 1.0) * 0.5);
          z.im = 0.0f;
        } else {
          z.re = -z.re;
          z.im = -z.im;
        }
        re = z.re;
        im = z.im;
      }
      split16_f(sp == 0 ? re : im, hh[2 * q], ll[2 * q]);          // K position 2l   (s = 0)
      split16_f(sp == 1 ? re : -im, hh[2 * q + 1], ll[2 * q + 1]);  // K position 2l+1 (s = 1)
    }
    *(uint4*)(th + j0) = *(const uint4*)hh;
    *(uint4*)(tl + j0) = *(const uint4*)ll;
  }
}

// Planes of the real embedding of op(X) (m x k complex; op: 0 = none, 2 = conjugate
// transpose): A (2m x 2k, row-major) = [[Re, -Im], [Im, Re]], the K axis interleaved
// by groups of 32 (complex column kk, part s at 64 (kk / 32) + 32 s + kk % 32), so that
// one 64-wide K-block holds both parts of 32 complex columns and a triangular operand
// spans a contiguous range of K-blocks.  32 x 32 tiles of op(X) staged in shared
// memory so both the read and the writes are coalesced; m and k multiples of 32.
// Grid (m / 32, k / 32, B), block (32, 8).
__global__ void __launch_bounds__(256) embed_a_kernel(const c32* __restrict__ X, int64_t ldx, int64_t sX, int op,
                                                      int m, int k, __half* Ah, __half* Al) {
  __shared__ c32 t[32][33];                       // t[row][col] of op(X)
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int64_t b = blockIdx.z;
  const c32* Xb = X + b * sX;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    if (op == 2) {
      c32 x = Xb[(c0 + tx) + (int64_t)(r0 + q) * ldx];
      x.im = -x.im;
      t[q][tx] = x;
    } else {
      t[tx][q] = Xb[(r0 + tx) + (int64_t)(c0 + q) * ldx];
    }
  }
  __syncthreads();
  const int64_t k2 = 2 * (int64_t)k;
  const int64_t base = b * 4 * (int64_t)m * k;
  for (int q = ty; q < 32; q += 8) {
    const c32 x = t[q][tx];
    const int64_t top = base + (int64_t)(r0 + q) * k2 + 2 * c0 + tx;
    const int64_t bot = top + (int64_t)m * k2;
    __half h, lo;
    split16_f(x.re, h, lo);
    Ah[top] = h; Al[top] = lo; Ah[bot + 32] = h; Al[bot + 32] = lo;
    split16_f(-x.im, h, lo);
    Ah[top + 32] = h; Al[top + 32] = lo;
    split16_f(x.im, h, lo);
    Ah[bot] = h; Al[bot] = lo;
  }
}

// The same planes as embed_a_kernel for k a multiple of 64: a 32 x 64 tile of op(X)
// staged in shared memory, then each thread writes the 8 K positions of one row and one
// group of 8 complex columns as 16-byte stores (Re, -Im on the top row, Im, Re on the
// bottom row, both planes).  Block (bx, by, b) of a grid (m / 32, k / 64, B), 256 threads.
__device__ __forceinline__ void embed_a64_block(const c32* __restrict__ X, int64_t ldx, int64_t sX, int op, int m,
                                                int k, __half* Ah, __half* Al, int bx, int by, int64_t b) {
  __shared__ c32 t[32][65];                       // t[row][col] of op(X)
  const int r0 = bx * 32, c0 = by * 64;
  const c32* Xb = X + b * sX;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  if (op == 2) {
    for (int q = ty; q < 32; q += 8) {            // lanes along the columns of op(X) (rows of X)
      c32 x0 = Xb[(c0 + tx) + (int64_t)(r0 + q) * ldx];
      c32 x1 = Xb[(c0 + 32 + tx) + (int64_t)(r0 + q) * ldx];
      x0.im = -x0.im;
      x1.im = -x1.im;
      t[q][tx] = x0;
      t[q][32 + tx] = x1;
    }
  } else {
    for (int q = ty; q < 64; q += 8) t[tx][q] = Xb[(r0 + tx) + (int64_t)(c0 + q) * ldx];
  }
  __syncthreads();
  const int r = tid >> 3, g = tid & 7;
  const int kk0 = c0 + 8 * g;                     // 8 complex columns inside one group of 32
  const int64_t k2 = 2 * (int64_t)k;
  const int64_t top = b * 4 * (int64_t)m * k + (int64_t)(r0 + r) * k2 + 64 * (kk0 / 32) + (kk0 % 32);
  const int64_t bot = top + (int64_t)m * k2;
  __align__(16) __half hre[8], lre[8], him[8], lim[8], hni[8], lni[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const c32 x = t[r][8 * g + e];
    split16_f(x.re, hre[e], lre[e]);
    split16_f(x.im, him[e], lim[e]);
    split16_f(-x.im, hni[e], lni[e]);
  }
  *(uint4*)(Ah + top) = *(const uint4*)hre;
  *(uint4*)(Al + top) = *(const uint4*)lre;
  *(uint4*)(Ah + top + 32) = *(const uint4*)hni;
  *(uint4*)(Al + top + 32) = *(const uint4*)lni;
  *(uint4*)(Ah + bot) = *(const uint4*)him;
  *(uint4*)(Al + bot) = *(const uint4*)lim;
  *(uint4*)(Ah + bot + 32) = *(const uint4*)hre;
  *(uint4*)(Al + bot + 32) = *(const uint4*)lre;
}

// The planes of embed_b_kernel for op(Y) = Y and k a multiple of 64, without staging:
// each thread reads 8 consecutive entries of one column of Y (64 bytes) and writes their
// Re and Im halves as 16-byte stores.  Block (bx, by, b) of a grid (k / 64, n / 32, B),
// 256 threads.
__device__ __forceinline__ void embed_b64_block(const c32* __restrict__ Y, int64_t ldy, int64_t sY, int k, int n,
                                                __half* Bh, __half* Bl, int bx, int by, int64_t b) {
  const int tid = threadIdx.x, g = tid & 7, jj = tid >> 3;
  const int kk0 = bx * 64 + 8 * g, j = by * 32 + jj;
  const float4* src = (const float4*)(Y + b * sY + kk0 + (int64_t)j * ldy);
  float4 v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = src[q];
  __align__(16) __half hre[8], lre[8], him[8], lim[8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    split16_f(v[q].x, hre[2 * q], lre[2 * q]);
    split16_f(v[q].y, him[2 * q], lim[2 * q]);
    split16_f(v[q].z, hre[2 * q + 1], lre[2 * q + 1]);
    split16_f(v[q].w, him[2 * q + 1], lim[2 * q + 1]);
  }
  const int64_t o = b * 2 * (int64_t)k * n + (int64_t)j * 2 * k + 64 * (kk0 / 32) + (kk0 % 32);
  *(uint4*)(Bh + o) = *(const uint4*)hre;
  *(uint4*)(Bl + o) = *(const uint4*)lre;
  *(uint4*)(Bh + o + 32) = *(const uint4*)him;
  *(uint4*)(Bl + o + 32) = *(const uint4*)lim;
}

__global__ void __launch_bounds__(256) embed_a64_kernel(const c32* __restrict__ X, int64_t ldx, int64_t sX, int op,
                                                        int m, int k, __half* Ah, __half* Al) {
  embed_a64_block(X, ldx, sX, op, m, k, Ah, Al, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Both operands' planes of one product in one launch: blocks [0, nA) of the flattened
// grid run embed_a64_block over (m / 32) x (k / 64) tiles, the rest embed_b64_block
// over (k / 64) x (n / 32); blockIdx.y is the trajectory.
__global__ void __launch_bounds__(256) embed_ab64_kernel(const c32* __restrict__ X, int64_t ldx, int64_t sX, int op,
                                                         const c32* __restrict__ Y, int64_t ldy, int64_t sY, int m,
                                                         int n, int k, __half* Ah, __half* Al, __half* Bh,
                                                         __half* Bl) {
  const int nAx = m / 32, nA = nAx * (k / 64), nBx = k / 64;
  const int i = blockIdx.x;
  if (i < nA) {
    embed_a64_block(X, ldx, sX, op, m, k, Ah, Al, i % nAx, i / nAx, blockIdx.y);
  } else {
    const int j = i - nA;
    embed_b64_block(Y, ldy, sY, k, n, Bh, Bl, j % nBx, j / nBx, blockIdx.y);
  }
}

// Planes of B (n x 2k, row-major): row j = the Re and Im parts of op(Y)[:, j], K
// interleaved by groups of 32 as in embed_a_kernel.  Grid (k / 32, n / 32, B),
// block (32, 8); k and n multiples of 32.
__global__ void __launch_bounds__(256) embed_b_kernel(const c32* __restrict__ Y, int64_t ldy, int64_t sY, int op,
                                                      int k, int n, __half* Bh, __half* Bl) {
  __shared__ c32 t[32][33];                       // t[j][kk] = op(Y)[kk][j]
  const int k0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int64_t b = blockIdx.z;
  const c32* Yb = Y + b * sY;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int q = ty; q < 32; q += 8) {
    if (op == 2) {
      c32 y = Yb[(j0 + tx) + (int64_t)(k0 + q) * ldy];
      y.im = -y.im;
      t[tx][q] = y;
    } else {
      t[q][tx] = Yb[(k0 + tx) + (int64_t)(j0 + q) * ldy];
    }
  }
  __syncthreads();
  const int64_t k2 = 2 * (int64_t)k;
  const int64_t base = b * 2 * (int64_t)k * n;
  for (int q = ty; q < 32; q += 8) {
    const c32 y = t[q][tx];
    const int64_t o = base + (int64_t)(j0 + q) * k2 + 2 * k0 + tx;
    __half h, lo;
    split16_f(y.re, h, lo);
    Bh[o] = h; Bl[o] = lo;
    split16_f(y.im, h, lo);
    Bh[o + 32] = h; Bl[o + 32] = lo;
  }
}

// Urm[(b L + i) 2N + c] = plane_b[i + L c] (V_b read as the L x 2N column-major
// matrix U~), both planes.  64 x 64 tiles: 16-byte loads along i and 16-byte stores
// along c.  In shared memory element (c, i) sits at column i ^ 8 (c >> 3) of row c, so
// the stores of a row's 8-element chunks and the gathers of 8 rows c = 8v .. 8v + 7 at
// one i both spread over all banks.  Grid (L / 64, 2N / 64, B), 256 threads.
__global__ void __launch_bounds__(256) transpose_planes_kernel(const __half* __restrict__ Vh,
                                                               const __half* __restrict__ Vl, int L, int N,
                                                               __half* Uh, __half* Ul, const int* cond) {
  if (cond && *cond == 0) return;
  __shared__ __align__(16) __half sh[64][64];
  __shared__ __align__(16) __half sl[64][64];
  const int i0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int64_t b = blockIdx.z;
  const int tid = threadIdx.x;
  const int64_t vb = b * 2 * (int64_t)L * N;
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int q = tid + 256 * hh, u = q & 7, c = q >> 3;
    const int64_t o = vb + (int64_t)(c0 + c) * L + i0 + 8 * u;
    const int col = (8 * u) ^ (8 * (c >> 3));
    *(uint4*)&sh[c][col] = *(const uint4*)(Vh + o);
    *(uint4*)&sl[c][col] = *(const uint4*)(Vl + o);
  }
  __syncthreads();
#pragma unroll
  for (int hh = 0; hh < 2; ++hh) {
    const int q = tid + 256 * hh, v = q & 7, i = q >> 3;
    __align__(16) __half oh[8], ol[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      oh[e] = sh[8 * v + e][i ^ (8 * v)];
      ol[e] = sl[8 * v + e][i ^ (8 * v)];
    }
    const int64_t o = (b * L + i0 + i) * 2 * (int64_t)N + c0 + 8 * v;
    *(uint4*)(Uh + o) = *(const uint4*)oh;
    *(uint4*)(Ul + o) = *(const uint4*)ol;
  }
}

// diag_b[k] = sum_s V_b[s,k]^2 (float64: 16-term float partial sums added into a
// double) and the same value on the diagonal of the complex64 Gram.  Replaces
// the tensor-core diagonal, whose fp32 accumulator loses up to one ulp per
// 16-deep MMA, biased toward zero on these all-positive sums.
// estat (second pass): the largest |diag_b[k] - 1| into estat[2b] as float bits.
__global__ void gram_diag_kernel(const float* __restrict__ V, int L, int N, int B, double* diag, c32* G,
                                 unsigned* estat, const int* cond) {
  if (cond && *cond == 0) return;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= (int64_t)B * N) return;
  const int64_t b = w / N, k = w % N;
  const float* col = V + b * 2 * (int64_t)L * N + k * 2 * (int64_t)L;
  double acc = 0.0;
  for (int s0 = 0; s0 < 2 * L; s0 += 32 * 16) {
    float part = 0.0f;
#pragma unroll 4
    for (int q = 0; q < 16; ++q) {
      const int s = s0 + q * 32 + lane;
      if (s < 2 * L) {
        const float x = col[s];
        part = fmaf(x, x, part);
      }
    }
    acc += (double)part;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    diag[b * N + k] = acc;
    G[b * (int64_t)N * N + k + k * (int64_t)N] = cmk((float)acc, 0.0f);
    if (estat) atomicMax(&estat[2 * b], __float_as_uint((float)fabs(acc - 1.0)));
  }
}

// The guard of the first-order second pass.  With G = 1 + E (E Hermitian), S the strict
// upper part of E and D its diagonal, the closed-form factor T = 1 - S - D/2 leaves
//   T^dag G T - 1 = -(F^dag F + F^2 + F^dag^2) + O(E^3),   F = S + D/2,
// whose entries are bounded by 3 (N o^2 + o d) + (3/4) d^2 (o = max |S|, d = max |D|).
// final == 0 (the second pass): flag = 1 when that bound exceeds tau for any trajectory,
// so the conditional extra pass runs; final != 0 (the extra pass, which measured the E
// the second pass left): a bound above tau means two closed-form passes were not enough
// (U ill-conditioned beyond the float Gram's reach), reported as FM_DEVERR_REORTH.
// Clears the statistics it read.  One warp.
__global__ void reorth_guard_kernel(unsigned* e, int B, int N, float tau, int final, int* flag,
                                    unsigned long long* counters, unsigned* seen, int* status) {
  const int lane = threadIdx.x;
  unsigned dmax = 0u, omax = 0u;
  int over = 0;
  for (int b = lane; b < B; b += 32) {
    const float d = __uint_as_float(e[2 * b]), o = __uint_as_float(e[2 * b + 1]);
    e[2 * b] = 0u;
    e[2 * b + 1] = 0u;
    const float bound = 3.0f * ((float)N * o * o + o * d) + 0.75f * d * d;
    over |= (bound > tau || !(bound == bound)) ? 1 : 0;
    dmax = max(dmax, __float_as_uint(d));
    omax = max(omax, __float_as_uint(o));
  }
  over = __any_sync(0xffffffffu, over);
  dmax = __reduce_max_sync(0xffffffffu, dmax);
  omax = __reduce_max_sync(0xffffffffu, omax);
  if (lane == 0) {
    const int k = final ? 2 : 0;
    seen[k] = max(seen[k], dmax);
    seen[k + 1] = max(seen[k + 1], omax);
    if (!final) {
      counters[0] += 1ull;
      if (over) counters[1] += 1ull;
      *flag = over;
    } else if (over && status) {
      atomicOr(status, FM_DEVERR_REORTH);
    }
  }
}

// dst = src (float4 words) unless cond is set and *cond == 0.
__global__ void copy_cond_kernel(const float4* __restrict__ src, float4* __restrict__ dst, int64_t n4,
                                 const int* cond) {
  if (cond && *cond == 0) return;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

struct MixedHost {
  int BN;
  int drain_kb;      // K-blocks between TMEM drains of the first-pass product that no second pass follows
  int n_prop, n_gram, n_trmm, n_trmm2;
  int4 *tiles_prop, *tiles_gram, *tiles_trmm, *tiles_trmm2;
  __half *urm_h, *urm_l;
  __half *ca_h, *ca_l, *cb_h, *cb_l;
  c32* xs;
  int64_t md;        // largest block dimension of the Cholesky recursion products
  c32 *gf, *rf, *tf, *dinvf, *xf;
  double* diag;
  GuardPtrs guard;
  CUtensorMap prop_Ah, prop_Al, prop_Bh, prop_Bl;
  CUtensorMap gram_Ah, gram_Al, gram_Bh, gram_Bl;
  CUtensorMap trmm_Ah, trmm_Al, trmm_Bh, trmm_Bl;
  CUtensorMap trmm2_Bh, trmm2_Bl;   // 256-row boxes of the factor planes (second pass)
  // block projective update
  bool pmb;
  int pb_kc;
  int *pb_list, *pb_count, *pb_pos;
  double* pb_ulist;
  __half *pb_wt_h, *pb_wt_l, *pb_dph, *pb_dpl, *pb_ath, *pb_atl, *pb_tth, *pb_ttl, *pb_xth, *pb_xtl;
  float *pb_dp, *pb_ap;
  PmbMats pm;
  std::vector<int> pb_hcount;
  // library streams of the first-pass Cholesky (parts of the batch side by side, the
  // first part on the step's stream)
  int nchains = 1;
  cudaStream_t cst[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[3] = {nullptr, nullptr, nullptr};
};

bool mixed_supported(int Lx, int Ly, int batch, int tile_config, std::string* why) {
  const int64_t L = (int64_t)Lx * Ly;
  if (L % 256 != 0) {
    *why = "mixed precision needs L = Lx*Ly divisible by 256 (N a multiple of 128)";
    return false;
  }
  if ((tile_config & ~0xff) || (tile_config & 3) == 3 || ((tile_config >> 5) & 3) == 3) {
    *why = "unknown tile_config bits";
    return false;
  }
  if ((tile_config & 3) == 2 && (L / 2) % 256 != 0) {
    *why = "tile width 256 needs N a multiple of 256";
    return false;
  }
  if ((int64_t)batch * L > (1ll << 31) / 4) {
    *why = "batch * L too large for the tensor maps";
    return false;
  }
  return true;
}

size_t mixed_scratch_bytes(int Lx, int Ly, int batch, int protocol) {
  return scratch_plan(Lx, Ly, batch, protocol).total;
}

void mixed_free(MixedHost* h) {
  if (!h) return;
  for (int i = 0; i < 3; ++i) {
    if (h->cst[i]) {
      cudaStreamSynchronize(h->cst[i]);
      cudaStreamDestroy(h->cst[i]);
    }
    if (h->join[i]) cudaEventDestroy(h->join[i]);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  delete h;
}

MixedHost* mixed_create(MixedCtx* c, std::string* why) {
  if (tc::configure_all() != cudaSuccess) {
    *why = "kernel attributes";
    return nullptr;
  }
  MixedHost* h = new MixedHost();
  const int L = c->L, N = c->N, B = c->B;
  h->BN = pick_bn(N, c->tile_config);
  h->drain_kb = 2 << ((c->tile_config >> 5) & 3);
  const int BN = h->BN;
  const int GM = pick_gm(c->tile_config);
  Scratch sp = scratch_plan(c->Lx, c->Ly, B, c->protocol);
  char* base = (char*)c->extra;
  h->tiles_prop = (int4*)(base + sp.tiles_prop);
  h->tiles_gram = (int4*)(base + sp.tiles_gram);
  h->tiles_trmm = (int4*)(base + sp.tiles_trmm);
  h->tiles_trmm2 = (int4*)(base + sp.tiles_trmm2);
  h->urm_h = (__half*)(base + sp.urm_h);
  h->urm_l = (__half*)(base + sp.urm_l);
  h->ca_h = (__half*)(base + sp.ca_h);
  h->ca_l = (__half*)(base + sp.ca_l);
  h->cb_h = (__half*)(base + sp.cb_h);
  h->cb_l = (__half*)(base + sp.cb_l);
  h->xs = (c32*)(base + sp.xs);
  h->md = N / 2 + 128;
  h->gf = (c32*)(base + sp.gf);
  h->rf = (c32*)(base + sp.rf);
  h->tf = (c32*)(base + sp.tf);
  h->dinvf = (c32*)(base + sp.dinvf);
  h->xf = (c32*)(base + sp.xf);
  h->diag = (double*)(base + sp.diag);
  h->guard = guard_ptrs(base + sp.guard, B);
  h->pmb = uses_pm_block(c->protocol, L, B);
  if (h->pmb) {
    const int64_t Kc = sp.pb_kc;
    h->pb_kc = sp.pb_kc;
    h->pb_list = (int*)(base + sp.pb_list);
    h->pb_ulist = (double*)(base + sp.pb_ulist);
    h->pb_count = (int*)(base + sp.pb_count);
    h->pb_pos = (int*)(base + sp.pb_pos);
    h->pb_wt_h = (__half*)(base + sp.pb_wt_h);
    h->pb_wt_l = (__half*)(base + sp.pb_wt_l);
    h->pb_dp = (float*)(base + sp.pb_dp);
    h->pb_dph = (__half*)(base + sp.pb_dph);
    h->pb_dpl = (__half*)(base + sp.pb_dpl);
    h->pb_ap = (float*)(base + sp.pb_ap);
    h->pb_ath = (__half*)(base + sp.pb_ath);
    h->pb_atl = (__half*)(base + sp.pb_atl);
    h->pb_tth = (__half*)(base + sp.pb_tth);
    h->pb_ttl = (__half*)(base + sp.pb_ttl);
    h->pb_xth = (__half*)(base + sp.pb_xth);
    h->pb_xtl = (__half*)(base + sp.pb_xtl);
    PmbMats& m = h->pm;
    m.Kc = (int)Kc;
    m.sM = Kc * Kc;
    m.sW = Kc * N;
    c32* mats = (c32*)(base + sp.pb_mats);
    m.C = mats;
    m.TBr = mats + 1 * B * m.sM;
    m.TBc = mats + 2 * B * m.sM;
    m.CTB = mats + 3 * B * m.sM;
    m.TA = mats + 4 * B * m.sM;
    m.CTA = mats + 5 * B * m.sM;
    m.TE = mats + 6 * B * m.sM;
    c32* vecs = (c32*)(base + sp.pb_vecs);
    m.rho = vecs;
    m.y = vecs + 1 * B * Kc;
    m.ys = vecs + 2 * B * Kc;
    m.g = vecs + 3 * B * Kc;
    m.ev = (PmbEvent*)(base + sp.pb_ev);
    m.Wc = (c32*)(base + sp.pb_wc);
    m.X = (c32*)(base + sp.pb_x);
    h->pb_hcount.assign(B, 0);
  }
  // chains of the first-pass Cholesky: two halves of the batch, or one trajectory per
  // chain up to four (tile_config bit 7, batches of three or more)
  h->nchains = B < 2 ? 1 : ((c->tile_config & FM_TILE_CHOL_CHAINS) && B >= 3 ? std::min(B, 4) : 2);
  bool streams_ok = h->nchains == 1 || cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; streams_ok && i + 1 < h->nchains; ++i)
    streams_ok = cudaStreamCreateWithFlags(&h->cst[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming) == cudaSuccess;
  if (!streams_ok) {
    *why = "Cholesky streams";
    mixed_free(h);
    return nullptr;
  }
  std::vector<int4> tp = tc::tile_list(2 * L / tc::BM, B * N / BN, 1, 1, false, BN, GM);
  std::vector<int4> tg = tc::tile_list(N / tc::BM, N / BN, B, 2, true, BN, GM);
  std::vector<int4> tt = tc::tile_list(L / tc::BM, 2 * N / 128, B, 1, false, 128, GM);
  std::vector<int4> tt2 = tc::tile_list(L / tc::BM, 2 * N / 256, B, 1, false, 256, GM);
  h->n_prop = (int)tp.size();
  h->n_gram = (int)tg.size();
  h->n_trmm = (int)tt.size();
  h->n_trmm2 = (int)tt2.size();
  bool ok = cudaMemcpyAsync(h->tiles_prop, tp.data(), tp.size() * 16, cudaMemcpyHostToDevice, c->st) == cudaSuccess &&
            cudaMemcpyAsync(h->tiles_gram, tg.data(), tg.size() * 16, cudaMemcpyHostToDevice, c->st) == cudaSuccess &&
            cudaMemcpyAsync(h->tiles_trmm, tt.data(), tt.size() * 16, cudaMemcpyHostToDevice, c->st) == cudaSuccess &&
            cudaMemcpyAsync(h->tiles_trmm2, tt2.data(), tt2.size() * 16, cudaMemcpyHostToDevice, c->st) ==
                cudaSuccess &&
            cudaMemsetAsync(base + sp.guard, 0, guard_bytes(B), c->st) == cudaSuccess &&
            cudaStreamSynchronize(c->st) == cudaSuccess;
  if (!ok) { *why = "tile upload"; mixed_free(h); return nullptr; }
  const uint64_t L2 = 2 * (uint64_t)L, N2 = 2 * (uint64_t)N;
  ok = tc::make_kmajor_map(&h->prop_Ah, c->Ah, L2, L2, L2, tc::BM) &&
       tc::make_kmajor_map(&h->prop_Al, c->Al, L2, L2, L2, tc::BM) &&
       tc::make_kmajor_map(&h->prop_Bh, c->Vh, L2, (uint64_t)B * N, L2, BN) &&
       tc::make_kmajor_map(&h->prop_Bl, c->Vl, L2, (uint64_t)B * N, L2, BN) &&
       tc::make_kmajor_map(&h->gram_Ah, c->Vh, L2, (uint64_t)B * N, L2, tc::BM) &&
       tc::make_kmajor_map(&h->gram_Al, c->Vl, L2, (uint64_t)B * N, L2, tc::BM) &&
       tc::make_kmajor_map(&h->gram_Bh, c->Vh, L2, (uint64_t)B * N, L2, BN) &&
       tc::make_kmajor_map(&h->gram_Bl, c->Vl, L2, (uint64_t)B * N, L2, BN) &&
       tc::make_kmajor_map(&h->trmm_Ah, h->urm_h, N2, (uint64_t)B * L, N2, tc::BM) &&
       tc::make_kmajor_map(&h->trmm_Al, h->urm_l, N2, (uint64_t)B * L, N2, tc::BM) &&
       tc::make_kmajor_map(&h->trmm_Bh, c->Th, N2, (uint64_t)B * N2, N2, 128) &&
       tc::make_kmajor_map(&h->trmm_Bl, c->Tl, N2, (uint64_t)B * N2, N2, 128) &&
       tc::make_kmajor_map(&h->trmm2_Bh, c->Th, N2, (uint64_t)B * N2, N2, 256) &&
       tc::make_kmajor_map(&h->trmm2_Bl, c->Tl, N2, (uint64_t)B * N2, N2, 256);
  if (!ok) { *why = "cuTensorMapEncodeTiled failed"; mixed_free(h); return nullptr; }
  return h;
}

namespace {

#define MCK(call)                                                   \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) {                                        \
      c->err = std::string(#call) + ": " + cudaGetErrorString(e_);  \
      return FM_ECUDA;                                              \
    }                                                               \
    c->launches += 1;                                               \
  } while (0)

// Operand shapes of cgemm_tc.
enum { CG_A_UPPER = 1, CG_A_LOWER = 2, CG_B_UPPER = 4, CG_HERM = 8 };

tc::Params base_params(MixedCtx* c, MixedHost* h) {
  tc::Params p;
  memset(&p, 0, sizeof(p));
  p.L = c->L;
  p.Ntraj = c->N;
  p.C = c->N / h->BN;
  p.status = c->status;
  return p;
}

// op(X) op(Y) on the tensor cores for complex64 blocks (all trajectories):
// C = alpha op(X) op(Y) + beta C, op(X) m x k, op(Y) k x n; m, n multiples of 128,
// k of 32.  The product runs as the real GEMM [[Re, -Im], [Im, Re]] (op X) x [Re; Im] (op Y).
// (Measured: even the 128-cubed products at the bottom of the recursion take ~7 us here
// plus their layout kernels, less than a CUDA-core complex64 GEMM of the same size.)
// shape: CG_A_UPPER / CG_A_LOWER (op(X) triangular, m == k) and CG_B_UPPER (op(Y) upper
// triangular, n == k) skip the K-blocks of zeros; CG_HERM (m == n, the result Hermitian)
// computes and writes only the tiles on or above the diagonal.  The skipped products are
// exact zeros, so the result is the full product's.
int cgemm_tc(MixedHost* h, MixedCtx* c, int opX, const c32* X, int64_t ldx, int64_t sX, int opY, const c32* Y,
             int64_t ldy, int64_t sY, int m, int n, int k, float alpha, float beta, c32* C, int64_t ldc,
             int64_t sC, int shape) {
  const int B = c->B;
  if (m % 128 || k % 32 || n % 128 || ((shape & (CG_A_UPPER | CG_A_LOWER)) && m != k) ||
      ((shape & CG_B_UPPER) && n != k) || ((shape & CG_HERM) && m != n)) {
    c->err = "cgemm sizes";
    return FM_EINVAL;
  }
  const bool y_aligned = ((uintptr_t)Y % 16 == 0) && (ldy % 2 == 0) && (sY % 2 == 0);
  if (k % 64 == 0 && opY == 0 && y_aligned) {
    const int nblk = (m / 32) * (k / 64) + (k / 64) * (n / 32);
    embed_ab64_kernel<<<dim3(nblk, B), 256, 0, c->st>>>(X, ldx, sX, opX, Y, ldy, sY, m, n, k, h->ca_h, h->ca_l,
                                                        h->cb_h, h->cb_l);
    MCK(cudaGetLastError());
  } else {
    if (k % 64 == 0) {
      embed_a64_kernel<<<dim3(m / 32, k / 64, B), 256, 0, c->st>>>(X, ldx, sX, opX, m, k, h->ca_h, h->ca_l);
    } else {
      embed_a_kernel<<<dim3(m / 32, k / 32, B), dim3(32, 8), 0, c->st>>>(X, ldx, sX, opX, m, k, h->ca_h, h->ca_l);
    }
    MCK(cudaGetLastError());
    embed_b_kernel<<<dim3(k / 32, n / 32, B), dim3(32, 8), 0, c->st>>>(Y, ldy, sY, opY, k, n, h->cb_h, h->cb_l);
    MCK(cudaGetLastError());
  }
  CUtensorMap ah, al, bh, bl;
  const uint64_t K2 = 2 * (uint64_t)k;
  if (!tc::make_kmajor_map(&ah, h->ca_h, K2, (uint64_t)B * 2 * m, K2, tc::BM) ||
      !tc::make_kmajor_map(&al, h->ca_l, K2, (uint64_t)B * 2 * m, K2, tc::BM) ||
      !tc::make_kmajor_map(&bh, h->cb_h, K2, (uint64_t)B * n, K2, 128) ||
      !tc::make_kmajor_map(&bl, h->cb_l, K2, (uint64_t)B * n, K2, 128)) {
    c->err = "cgemm tensor maps";
    return FM_ECUDA;
  }
  tc::Params p = base_params(c, h);
  p.tiles = nullptr;
  p.mtiles = 2 * m / tc::BM;
  p.ntiles_n = n / 128;
  p.ntiles = B * p.mtiles * p.ntiles_n;
  p.kblocks = 2 * k / tc::BK;
  p.a_rows_per_b = 2 * m;
  p.b_rows_per_b = n;
  // the epilogue writes C = alpha (D_re + i D_im) + beta C itself (tiles below the diagonal
  // of a Hermitian product are neither computed nor written)
  p.mode = tc::MODE_CPLX;
  p.out_c = (float*)C;
  p.ld_out = ldc;
  p.out_batch_stride = sC;
  p.alpha = alpha;
  p.beta = beta;
  // K-block = 32 complex columns; a 128-row (column) tile spans 4 of them
  p.mt_mod = m / tc::BM;
  p.kb_lo_mt = (shape & CG_A_UPPER) ? 4 : 0;
  p.kb_hi_mt = (shape & CG_A_LOWER) ? 4 : 0;
  p.kb_hi_nt = (shape & CG_B_UPPER) ? 4 : 0;
  p.herm_upper = (shape & CG_HERM) ? 1 : 0;
  // balanced orders for the triangular and Hermitian shapes (their tiles' K ranges or
  // counts differ by row or column; the plain raster left CTAs up to 1.4 x the mean)
  const int M = m / tc::BM;
  if ((shape & (CG_A_UPPER | CG_A_LOWER)) && M % 2 == 0) {
    p.order = tc::ORDER_PAIRS_A;
  } else if ((shape & CG_B_UPPER) && p.ntiles_n % 2 == 0) {
    p.order = tc::ORDER_PAIRS_B;
  } else if (shape & CG_HERM) {
    p.order = tc::ORDER_HERM;
    p.ntiles = B * M * (M + 1);
  }
  // with the batch factored as parts side by side, a product that fills the GPU leaves 8 SMs
  // to the other parts' latency-bound leaves and small products (its CTAs hold their SMs
  // for the whole launch)
  const int sms = tc::sm_count();
  const int grid = h->nchains >= 2 && p.ntiles > sms && sms > 32 ? sms - 8 : sms;
  MCK(tc::launch(c->st, 128, ah, al, bh, bl, p, grid));
  return FM_OK;
}

// R and T = R^-1 of the n x n diagonal block at `off` of G (= R^dag R), recursively,
// on the complex64 copies (the first pass only needs its factor to bring U within
// reach of the second, float64-factored pass):
//   R11, T11 <- block(off, h);  R12 = T11^dag G12;  G22 -= R12^dag R12;
//   R22, T22 <- block(off + h, n - h);  T12 = -T11 (R12 T22).
// Blocks of <= 128 are factored on the CUDA cores; the products run on the tensor cores,
// each skipping the zero half of its triangular operand, and the Hermitian update of
// G22 computes its upper tiles only (nothing reads below the diagonal of G).
int chol_inv_rec(MixedHost* h, MixedCtx* c, int off, int n) {
  const int N = c->N;
  const int64_t sNN = (int64_t)N * N;
  c32* G = h->gf;
  c32* R = h->rf;
  c32* T = h->tf;
  const int64_t d0 = off + (int64_t)off * N;
  if (n <= 128) {
    MCK(chol_inv_leaf(c->st, G + d0, R + d0, T + d0, n, N, sNN, c->B, c->status));
    return FM_OK;
  }
  const int hh = std::max(128, (n / 2 / 128) * 128);
  const int m2 = n - hh;
  const int64_t o12 = off + (int64_t)(off + hh) * N, d1 = (off + hh) + (int64_t)(off + hh) * N;
  int r;
  const int64_t sXS = (int64_t)h->md * h->md;  // batch stride of the xs scratch
  if ((r = chol_inv_rec(h, c, off, hh))) return r;
  if ((r = cgemm_tc(h, c, 2, T + d0, N, sNN, 0, G + o12, N, sNN, hh, m2, hh, 1.f, 0.f, R + o12, N, sNN,
                    CG_A_LOWER)))
    return r;
  if ((r = cgemm_tc(h, c, 2, R + o12, N, sNN, 0, R + o12, N, sNN, m2, m2, hh, -1.f, 1.f, G + d1, N, sNN, CG_HERM)))
    return r;
  if ((r = chol_inv_rec(h, c, off + hh, m2))) return r;
  if ((r = cgemm_tc(h, c, 0, R + o12, N, sNN, 0, T + d1, N, sNN, hh, m2, m2, 1.f, 0.f, h->xs, hh, sXS, CG_B_UPPER)))
    return r;
  if ((r = cgemm_tc(h, c, 0, T + d0, N, sNN, 0, h->xs, hh, sXS, hh, m2, hh, -1.f, 0.f, T + o12, N, sNN,
                    CG_A_UPPER)))
    return r;
  return FM_OK;
}

// The first-pass factorisation of the whole batch as parts side by side (two halves, or
// one trajectory per part up to four): the parts' recursions are independent, so one
// part's latency-bound leaves (a CTA per trajectory) and small products run while the
// others' products fill the GPU.  Part i works on its trajectories' slices of the factor
// and operand scratch (per-trajectory strides), part 0 on the step's stream and the others
// on library streams forked from it and joined back into it (a captured graph holds all).
// Every tile and every leaf is one trajectory's, so the split changes no result.
int chol_chains(MixedHost* h, MixedCtx* c) {
  const int B = c->B, P = std::min(h->nchains, B);
  if (P < 2) return chol_inv_rec(h, c, 0, c->N);
  const int64_t sNN = (int64_t)c->N * c->N, md2 = h->md * h->md;
  if (cudaEventRecord(h->fork, c->st) != cudaSuccess) {
    c->err = "Cholesky stream fork";
    return FM_ECUDA;
  }
  for (int i = 1; i < P; ++i)
    if (cudaStreamWaitEvent(h->cst[i - 1], h->fork, 0) != cudaSuccess) {
      c->err = "Cholesky stream fork";
      return FM_ECUDA;
    }
  int r = FM_OK, b0 = 0;
  for (int i = 0; i < P; ++i) {
    const int nb = B / P + (i < B % P ? 1 : 0);
    MixedHost hp = *h;                         // the copy owns nothing
    hp.gf += b0 * sNN;
    hp.rf += b0 * sNN;
    hp.tf += b0 * sNN;
    hp.ca_h += b0 * 4 * md2;
    hp.ca_l += b0 * 4 * md2;
    hp.cb_h += b0 * 2 * md2;
    hp.cb_l += b0 * 2 * md2;
    hp.xs += b0 * md2;
    hp.pb_hcount.clear();
    MixedCtx cp = *c;
    cp.B = nb;
    cp.st = i == 0 ? c->st : h->cst[i - 1];
    cp.launches = 0;
    if (r == FM_OK) {
      r = chol_inv_rec(&hp, &cp, 0, c->N);
      if (r) c->err = cp.err;
    }
    c->launches += cp.launches;
    b0 += nb;
  }
  // join even after an error, so that the step's stream never runs ahead of a part
  bool joined = true;
  for (int i = 1; i < P; ++i)
    joined = cudaEventRecord(h->join[i - 1], h->cst[i - 1]) == cudaSuccess &&
             cudaStreamWaitEvent(c->st, h->join[i - 1], 0) == cudaSuccess && joined;
  if (r) return r;
  if (!joined) {
    c->err = "Cholesky stream join";
    return FM_ECUDA;
  }
  return FM_OK;
}

// Target of the second-pass guard: the bound on the entries of U^dag U - 1 that the
// first-order factor may leave (a tenth of the 1e-6 orthonormality bar).
constexpr float kReorthTau = 1e-7f;

// One CholeskyQR pass on V: Gram (tensor) -> inverse factor -> U <- U + U (T - 1) (tensor).
// first == true: T = R^-1 from the recursive factorisation (G far from 1), and
//   the product accumulates in fp32 registers every 2 K-blocks;
// first == false: G = 1 + E with |E| small after a full pass, T = 1 - F to first
//   order (O(|E|^2) error), F built from G with its float64 diagonal; the Gram's
//   epilogue and diagonal kernel record the largest entries of E for the guard
//   (reorth_guard_kernel).
// how a pass leaves the state: PASS_SWAP the product in V2, then V and V2 swap (host
// pointers); PASS_EXTRA a closed-form pass run only when the guard's device flag is set
// (every launch returns at once when it is clear), the product copied back into V;
// PASS_INPLACE the product copied back into V unconditionally.  The last two keep the
// buffers where a captured step graph expects them.
enum PassMode { PASS_SWAP = 0, PASS_EXTRA = 1, PASS_INPLACE = 2 };

int qr_pass(MixedHost* h, MixedCtx* c, bool first, bool paired, int mode = PASS_SWAP) {
  const int L = c->L, N = c->N, B = c->B, BN = h->BN;
  const int grid = tc::sm_count();
  const bool extra = mode == PASS_EXTRA;
  const int* cond = extra ? h->guard.flag : nullptr;
  unsigned* estat = first ? nullptr : (extra ? h->guard.e3 : h->guard.e2);
  tc::Params p = base_params(c, h);
  p.mode = tc::MODE_GRAM;
  p.ntiles = h->n_gram;
  p.tiles = h->tiles_gram;
  p.kblocks = 2 * L / tc::BK;
  p.a_rows_per_b = N;
  p.b_rows_per_b = N;
  p.k_shift = L;
  p.kdim = 2 * L;
  p.out_gf = (float*)h->gf;
  p.estat = estat;
  p.cond = cond;
  c->timer->begin(FM_PH_GRAM);
  MCK(tc::launch(c->st, BN, h->gram_Ah, h->gram_Al, h->gram_Bh, h->gram_Bl, p, grid));
  gram_diag_kernel<<<FM_CEIL_DIV((int64_t)B * N * 32, 256), 256, 0, c->st>>>(c->V, L, N, B, h->diag, h->gf, estat,
                                                                             cond);
  MCK(cudaGetLastError());
  if (!first) {
    reorth_guard_kernel<<<1, 32, 0, c->st>>>(estat, B, N, kReorthTau, extra ? 1 : 0, h->guard.flag,
                                             h->guard.counters, h->guard.seen, c->status);
    MCK(cudaGetLastError());
  }
  c->timer->end(FM_PH_GRAM);
  c->timer->begin(FM_PH_CHOLESKY);
  if (first) {
    int r = chol_chains(h, c);
    if (r) return r;
  }
  build_ttilde_kernel<<<(unsigned)(2 * (int64_t)B * N), 256, 0, c->st>>>(first ? h->tf : h->gf, h->diag,
                                                                          first ? 0 : 1, N, c->Th, c->Tl, cond);
  MCK(cudaGetLastError());
  transpose_planes_kernel<<<dim3(L / 64, 2 * N / 64, B), 256, 0, c->st>>>(c->Vh, c->Vl, L, N, h->urm_h,
                                                                                  h->urm_l, cond);
  MCK(cudaGetLastError());
  c->timer->end(FM_PH_CHOLESKY);
  // first pass: 128-wide tiles (fp32 register accumulation every 2 K-blocks when no
  // second pass follows); second pass: tiles of the state's width accumulated in TMEM
  // (128: two accumulator sets, the epilogue overlapping the next tile)
  const bool wide2 = !first && h->BN == 256;
  p = base_params(c, h);
  p.mode = tc::MODE_TRMM;
  p.ntiles = wide2 ? h->n_trmm2 : h->n_trmm;
  p.tiles = wide2 ? h->tiles_trmm2 : h->tiles_trmm;
  p.kblocks = 2 * N / tc::BK;
  p.tri_k = 1;
  p.a_rows_per_b = L;
  p.b_rows_per_b = 2 * N;
  p.out_f = c->V2;
  p.out_h = c->Vh;
  p.out_l = c->Vl;
  p.in_f = c->V;
  p.cond = cond;
  // the first pass drains TMEM into fp32 registers every drain_kb K-blocks (2 by default,
  // fm_params.tile_config bits 5-6) when its result stays the state until the next step
  // (the fp32 TMEM accumulators round toward zero: up to ~1e-4 relative over 16384 terms);
  // when the second pass follows at once it removes that error with the rest (to
  // O(|E|^2) ~ 1e-8), so the plain kernel serves
  p.chunk_kb = (first && !paired) ? h->drain_kb : 0;
  c->timer->begin(FM_PH_TRMM);
  if (wide2) MCK(tc::launch(c->st, 256, h->trmm_Ah, h->trmm_Al, h->trmm2_Bh, h->trmm2_Bl, p, grid));
  else MCK(tc::launch(c->st, 128, h->trmm_Ah, h->trmm_Al, h->trmm_Bh, h->trmm_Bl, p, grid));
  if (mode != PASS_SWAP) {
    const int64_t n4 = (int64_t)B * 2 * L * N / 4;
    copy_cond_kernel<<<(unsigned)std::min<int64_t>(FM_CEIL_DIV(n4, 256), 8 * grid), 256, 0, c->st>>>(
        (const float4*)c->V2, (float4*)c->V, n4, cond);
    MCK(cudaGetLastError());
  }
  c->timer->end(FM_PH_TRMM);
  if (mode == PASS_SWAP) std::swap(c->V, c->V2);
  return FM_OK;
}

// The second (closed-form) pass and, when its guard asks for it, one more.
int second_pass(MixedHost* h, MixedCtx* c, int mode = PASS_SWAP) {
  int r = qr_pass(h, c, false, true, mode);
  if (r) return r;
  return qr_pass(h, c, false, true, PASS_EXTRA);
}

// Tensor-core product D = A B^T of K-major fp16 planes (raster tile order, one
// batch item): A rows M, B rows Nd, contraction Kd; mode PLAIN (D into out_f with
// ld_out) or ADDV (out_f = in_f + D and its planes).
int plane_gemm(MixedHost* h, MixedCtx* c, int mode, const __half* ah, const __half* al, const __half* bh,
               const __half* bl, int M, int Nd, int Kd, int BN, int batch, float* out_f, int64_t ld_out,
               int64_t out_stride, const float* in_f, __half* out_h, __half* out_l) {
  CUtensorMap mah, mal, mbh, mbl;
  const uint64_t Mb = (uint64_t)M * batch, Nb = (uint64_t)Nd * batch;
  if (!tc::make_kmajor_map(&mah, ah, Kd, Mb, Kd, tc::BM) || !tc::make_kmajor_map(&mal, al, Kd, Mb, Kd, tc::BM) ||
      !tc::make_kmajor_map(&mbh, bh, Kd, Nb, Kd, BN) || !tc::make_kmajor_map(&mbl, bl, Kd, Nb, Kd, BN)) {
    c->err = "block projective update: tensor maps";
    return FM_ECUDA;
  }
  tc::Params p = base_params(c, h);
  p.mode = mode;
  p.tiles = nullptr;
  p.mtiles = M / tc::BM;
  p.ntiles_n = Nd / BN;
  p.ntiles = p.mtiles * p.ntiles_n * batch;
  p.a_rows_per_b = M;
  p.b_rows_per_b = Nd;
  p.out_batch_stride = out_stride;
  p.kblocks = Kd / tc::BK;
  p.out_f = out_f;
  p.ld_out = ld_out;
  p.in_f = in_f;
  p.out_h = out_h;
  p.out_l = out_l;
  MCK(tc::launch(c->st, BN, mah, mal, mbh, mbl, p, tc::sm_count()));
  return FM_OK;
}

// The projective measurements of the step as one block (pm_block.cu): select
// the sites, form P = U0 W^dag and C on the tensor cores, run the events on the
// K x K coefficients, then U <- U0 + A B^dag on the tensor cores.  *done =
// false (nothing changed) when a trajectory selected more sites than the
// block scratch holds; the caller then takes the per-event path.
int pm_block_step(MixedHost* h, MixedCtx* c, bool* done) {
  const int L = c->L, N = c->N, B = c->B;
  *done = false;
  pm_args a;
  a.U = c->V; a.L = L; a.N = N; a.batch = B; a.layout = 1;
  a.gamma = c->gamma; a.dt = c->dt; a.traj = c->traj; a.step = c->step; a.seed = c->seed;
  a.force = c->force; a.force_n = c->force_n;
  MCK(pm_select(c->st, a, h->pb_list, h->pb_ulist, h->pb_count));
  int* hc = h->pb_hcount.data();
  MCK(cudaMemcpyAsync(hc, h->pb_count, sizeof(int) * B, cudaMemcpyDeviceToHost, c->st));
  MCK(cudaStreamSynchronize(c->st));
  int kmax = 0;
  for (int b = 0; b < B; ++b) kmax = std::max(kmax, hc[b]);
  if (kmax > h->pb_kc) return FM_OK;
  *done = true;
  if (kmax == 0) return FM_OK;
  const int K = ((kmax + 63) / 64) * 64;
  const int Kc = h->pb_kc;
  PmbMats& m = h->pm;
  const int64_t sD = (int64_t)L * 2 * K;          // per-trajectory stride of the L x 2K arrays
  // U~ planes (L x 2N per trajectory, K-major) of the propagated state (the
  // propagation writes the float state only, so its planes are made here)
  MCK(split_planes(c->st, c->V, c->Vh, c->Vl, (int64_t)B * 2 * L * N));
  transpose_planes_kernel<<<dim3(L / 64, 2 * N / 64, B), 256, 0, c->st>>>(c->Vh, c->Vl, L, N, h->urm_h,
                                                                                  h->urm_l, nullptr);
  MCK(cudaGetLastError());
  MCK(pmb_setup(c->st, h->pb_list, h->pb_count, L, B, kmax, h->pb_pos));
  MCK(cudaMemsetAsync(m.C, 0, sizeof(c32) * 7 * (size_t)B * m.sM, c->st));
  // P_b = U0_b W_b^dag as the row-major real form [Re P | Im P] (L x 2K), all trajectories
  MCK(pmb_gather_w(c->st, h->urm_h, h->urm_l, L, N, h->pb_list, h->pb_count, B, K, h->pb_wt_h, h->pb_wt_l));
  int r = plane_gemm(h, c, tc::MODE_PLAIN, h->pb_wt_h, h->pb_wt_l, h->urm_h, h->urm_l, 2 * K, L, 2 * N, 256, B,
                     h->pb_dp, 2 * K, sD, nullptr, nullptr, nullptr);
  if (r) return r;
  MCK(pmb_gather_c(c->st, h->pb_dp, sD, L, K, B, h->pb_list, h->pb_count, m));
  // the events, in order: many trajectories or few events in one launch (one CTA per
  // trajectory); else one launch per phase of each event, spread over the GPU
  if (pmb_events_fit(B, kmax)) {
    MCK(pmb_events(c->st, Kc, L, B, h->pb_count, h->pb_list, h->pb_ulist, c->step, m, c->log,
                   (unsigned long long*)c->log_count, c->log_capacity));
  } else {
    for (int i = 0; i < kmax; ++i) {
      MCK(pmb_event(c->st, i, Kc, L, B, h->pb_count, h->pb_list, h->pb_ulist, c->step, m, c->log,
                    (unsigned long long*)c->log_count, c->log_capacity, kmax));
      c->launches += i > 0 ? 3 : 2;               // with the one MCK counts: 4 (3 for the first event)
    }
  }
  // B^dag = T_B^dag W
  MCK(pmb_gather_wc(c->st, c->V, L, N, K, B, h->pb_list, h->pb_count, m));
  const c32 one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
  MCK(zgemm<float>(c->st, K, N, K, OP_C, OP_N, one, m.TBc, Kc, m.sM, m.Wc, Kc, m.sW, zero, m.X, Kc, m.sW, B, 0));
  // A = P T_A (+ E_S T_E in the planes), then V2_b = V_b + A B^dag, all trajectories
  MCK(pmb_ttilde(c->st, m, K, B, h->pb_tth, h->pb_ttl));
  MCK(pmb_split(c->st, h->pb_dp, (int64_t)B * L * 2 * K, h->pb_dph, h->pb_dpl));
  r = plane_gemm(h, c, tc::MODE_PLAIN, h->pb_tth, h->pb_ttl, h->pb_dph, h->pb_dpl, 2 * K, L, 2 * K, 256, B,
                 h->pb_ap, 2 * K, sD, nullptr, nullptr, nullptr);
  if (r) return r;
  MCK(pmb_atilde(c->st, h->pb_ap, L, K, B, h->pb_pos, m, h->pb_ath, h->pb_atl));
  MCK(pmb_xtilde(c->st, m, K, B, N, h->pb_xth, h->pb_xtl));
  const int BNu = (N % 256 == 0) ? 256 : 128;
  r = plane_gemm(h, c, tc::MODE_ADDV, h->pb_ath, h->pb_atl, h->pb_xth, h->pb_xtl, 2 * L, N, 2 * K, BNu, B, c->V2,
                 2 * L, (int64_t)2 * L * N, c->V, c->Vh, c->Vl);
  if (r) return r;
  std::swap(c->V, c->V2);
  return FM_OK;
}

}  // namespace

int mixed_guard_stats(MixedHost* h, cudaStream_t st, int64_t* counts, double* maxima) {
  unsigned char buf[32];
  if (cudaMemcpyAsync(buf, h->guard.counters, 32, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return FM_ECUDA;
  unsigned long long cnt[2];
  unsigned seen[4];
  memcpy(cnt, buf, 16);
  memcpy(seen, buf + 16, 16);
  counts[0] = (int64_t)cnt[0];
  counts[1] = (int64_t)cnt[1];
  for (int i = 0; i < 4; ++i) {
    float f;
    memcpy(&f, &seen[i], 4);
    maxima[i] = (double)f;
  }
  // the maxima restart from zero; the counters keep counting
  if (cudaMemsetAsync(h->guard.seen, 0, 16, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return FM_ECUDA;
  return FM_OK;
}

int mixed_settle(MixedHost* h, MixedCtx* c) { return second_pass(h, c, PASS_INPLACE); }

int mixed_reorth(MixedHost* h, MixedCtx* c) {
  const int L = c->L, N = c->N, B = c->B;
  MCK(split_planes(c->st, c->V, c->Vh, c->Vl, (int64_t)B * 2 * L * N));
  int r = qr_pass(h, c, true, true);
  if (r) return r;
  return second_pass(h, c);
}

int mixed_step(MixedHost* h, MixedCtx* c) {
  const int L = c->L, N = c->N, B = c->B, BN = h->BN;
  const int grid = tc::sm_count();
  if (c->protocol == FM_HOMODYNE_RK4) {
    // App. A's integrator: <n> of U(t), the weights' logarithms, four Horner stages
    const int nch = occupation_chunks(L, N, B);
    c->timer->begin(FM_PH_MEASURE);
    MCK(rownorm_partials_v(c->st, c->V, L, N, B, c->part, nch));
    MCK(reduce_occupations(c->st, c->part, nch, L, B, c->nocc, c->w, c->gamma, c->dt, c->traj, c->step, c->seed));
    c->timer->end(FM_PH_MEASURE);
    c->timer->begin(FM_PH_PROPAGATE);
    const double hJ = c->dt * c->J;
    MCK(rk4_stage(c->st, 1, c->V, c->V, c->rk4buf, L, N, B, c->Lx, c->Ly, c->w, hJ, 0.25));
    MCK(rk4_stage(c->st, 1, c->V, c->rk4buf, c->V2, L, N, B, c->Lx, c->Ly, c->w, hJ, 1.0 / 3.0));
    MCK(rk4_stage(c->st, 1, c->V, c->V2, c->rk4buf, L, N, B, c->Lx, c->Ly, c->w, hJ, 0.5));
    MCK(rk4_stage(c->st, 1, c->V, c->rk4buf, c->V2, L, N, B, c->Lx, c->Ly, c->w, hJ, 1.0));
    std::swap(c->V, c->V2);
    MCK(split_planes(c->st, c->V, c->Vh, c->Vl, (int64_t)B * 2 * L * N));
    c->timer->end(FM_PH_PROPAGATE);
    const bool second = (c->global_step + 1) % c->reorth_interval == 0;
    int r = qr_pass(h, c, true, second);
    if (r) return r;
    if (second && (r = second_pass(h, c))) return r;
    MCK(bump_steps(c->st, c->step, B));
    return FM_OK;
  }
  // 1. propagation V2 = A V with row sums of squares
  int nchunks = 2 * (N / BN);
  c->timer->begin(FM_PH_PROPAGATE);
  if (c->prop_banded) {
    // stencils along x (and y): V -> V2 (-> V); the last pass sums |U|^2 per row
    const bool torus = c->Ly > 1;
    const int nx = band_chunks(c->Lx, c->Ly, N, B, 0, 1), ny = band_chunks(c->Lx, c->Ly, N, B, 1, 1);
    nchunks = torus ? ny : nx;                     // chunks of the pass that sums |U|^2 per row
    MCK(band_propagate(c->st, 1, c->V, c->V2, L, N, B, c->Lx, c->Ly, 0, c->band_tx, c->band_ox, c->ntap_x,
                       torus ? nullptr : c->part, nx));
    if (torus) {
      MCK(band_propagate(c->st, 1, c->V2, c->V, L, N, B, c->Lx, c->Ly, 1, c->band_ty, c->band_oy, c->ntap_y,
                         c->part, ny));
    } else {
      std::swap(c->V, c->V2);
    }
  } else {
    tc::Params p = base_params(c, h);
    p.mode = tc::MODE_PROP;
    p.ntiles = h->n_prop;
    p.tiles = h->tiles_prop;
    p.kblocks = 2 * L / tc::BK;
    p.out_f = c->V2;
    p.ld_out = 2 * (int64_t)L;
    p.partial = c->part;
    MCK(tc::launch(c->st, BN, h->prop_Ah, h->prop_Al, h->prop_Bh, h->prop_Bl, p, grid));
    std::swap(c->V, c->V2);
  }
  c->timer->end(FM_PH_PROPAGATE);
  const int k = c->reorth_interval;
  if (c->protocol == FM_HOMODYNE) {
    c->timer->begin(FM_PH_MEASURE);
    MCK(reduce_occupations(c->st, c->part, nchunks, L, B, c->nocc, c->w, c->gamma, c->dt, c->traj, c->step, c->seed));
    MCK(scale_rows_v(c->st, c->V, c->Vh, c->Vl, L, N, B, c->w));
    c->timer->end(FM_PH_MEASURE);
    const bool second = (c->global_step + 1) % k == 0;
    int r = qr_pass(h, c, true, second);
    if (r) return r;
    if (second) {
      r = second_pass(h, c);
      if (r) return r;
    }
  } else {
    pm_args a;
    a.U = c->V; a.L = L; a.N = N; a.batch = B; a.layout = 1;
    a.gamma = c->gamma; a.dt = c->dt; a.traj = c->traj; a.step = c->step; a.seed = c->seed;
    a.xbuf = c->xbuf; a.vbuf = c->vbuf;
    a.log = c->log; a.log_count = c->log_count; a.log_capacity = c->log_capacity;
    a.dev_status = c->status;
    a.force = c->force; a.force_n = c->force_n;
    c->timer->begin(FM_PH_MEASURE);
    bool done = false;
    if (h->pmb) {
      int r = pm_block_step(h, c, &done);
      if (r) return r;
    }
    if (!done) {
      a.U = c->V;
      if (pm_use_wide(L, N, B)) {
        cudaError_t e = pm_measure_wide(c->st, a, c->pmw, &c->launches);
        if (e != cudaSuccess) { c->err = std::string("projective update: ") + cudaGetErrorString(e); return FM_ECUDA; }
      } else {
        MCK(pm_measure(c->st, a));
      }
      MCK(split_planes(c->st, c->V, c->Vh, c->Vl, (int64_t)B * 2 * L * N));
    }
    c->timer->end(FM_PH_MEASURE);
    if ((c->global_step + 1) % k == 0) {
      int r = qr_pass(h, c, true, true);
      if (r) return r;
      r = second_pass(h, c);
      if (r) return r;
    }
  }
  MCK(bump_steps(c->st, c->step, B));
  return FM_OK;
}

}  // namespace fm

// ====================================================================== test hooks
using namespace fm;

extern "C" int fmx_tc_gemm(const void* Ah, const void* Al, const void* Bh, const void* Bl, int M, int N, int K,
                           float* D, int BN, int grid, int chunk_kb, int raster, void* d_tiles, void* stream) {
  if (M % tc::BM || (BN != 128 && BN != 256) || N % BN || K % tc::BK) return (int)cudaErrorInvalidValue;
  if (chunk_kb > 0 && BN != 128) return (int)cudaErrorInvalidValue;
  CUtensorMap a_h, a_l, b_h, b_l;
  if (!tc::make_kmajor_map(&a_h, (const __half*)Ah, K, M, K, tc::BM) ||
      !tc::make_kmajor_map(&a_l, (const __half*)Al, K, M, K, tc::BM) ||
      !tc::make_kmajor_map(&b_h, (const __half*)Bh, K, N, K, BN) ||
      !tc::make_kmajor_map(&b_l, (const __half*)Bl, K, N, K, BN))
    return (int)cudaErrorInvalidValue;
  cudaStream_t st = (cudaStream_t)stream;
  tc::Params p;
  memset(&p, 0, sizeof(p));
  p.mode = tc::MODE_PLAIN;
  p.mtiles = M / tc::BM;
  p.ntiles_n = N / BN;
  p.ntiles = p.mtiles * p.ntiles_n;
  if (raster) {
    p.tiles = nullptr;
  } else {
    std::vector<int4> t = tc::tile_list(M / tc::BM, N / BN, 1, 1, false, BN, 16);
    cudaError_t e = cudaMemcpyAsync(d_tiles, t.data(), t.size() * 16, cudaMemcpyHostToDevice, st);
    if (e) return (int)e;
    p.tiles = (const int4*)d_tiles;
  }
  p.kblocks = K / tc::BK;
  p.chunk_kb = chunk_kb > 0 ? chunk_kb : 0;
  p.out_f = D;
  p.ld_out = M;
  return (int)tc::launch(st, BN, a_h, a_l, b_h, b_l, p, grid);
}

extern "C" int fmx_tc_gram(const void* Vh, const void* Vl, int L, int N, int B, float* G, int BN, void* d_tiles,
                           void* stream) {
  if (N % tc::BM || (BN != 128 && BN != 256) || N % BN || (2 * L) % tc::BK) return (int)cudaErrorInvalidValue;
  CUtensorMap a_h, a_l, b_h, b_l;
  const uint64_t L2 = 2 * (uint64_t)L;
  if (!tc::make_kmajor_map(&a_h, (const __half*)Vh, L2, (uint64_t)B * N, L2, tc::BM) ||
      !tc::make_kmajor_map(&a_l, (const __half*)Vl, L2, (uint64_t)B * N, L2, tc::BM) ||
      !tc::make_kmajor_map(&b_h, (const __half*)Vh, L2, (uint64_t)B * N, L2, BN) ||
      !tc::make_kmajor_map(&b_l, (const __half*)Vl, L2, (uint64_t)B * N, L2, BN))
    return (int)cudaErrorInvalidValue;
  std::vector<int4> t = tc::tile_list(N / tc::BM, N / BN, B, 2, true, BN, 16);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(d_tiles, t.data(), t.size() * 16, cudaMemcpyHostToDevice, st);
  if (e) return (int)e;
  tc::Params p;
  memset(&p, 0, sizeof(p));
  p.mode = tc::MODE_GRAM;
  p.ntiles = (int)t.size();
  p.tiles = (const int4*)d_tiles;
  p.kblocks = 2 * L / tc::BK;
  p.a_rows_per_b = N;
  p.b_rows_per_b = N;
  p.k_shift = L;
  p.kdim = 2 * L;
  p.out_gf = G;
  p.L = L;
  p.Ntraj = N;
  return (int)tc::launch(st, BN, a_h, a_l, b_h, b_l, p, tc::sm_count());
}
