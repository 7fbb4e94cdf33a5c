// Gram matrix of the subsystem block for the entanglement-entropy eigenproblem
// (Sec. II), M = Y Y^dag, on the tensor cores with exact products.
//
// Y is the block of gathered rows of U_A (n x N, the sites of A) when n <= N,
// else its transpose (N x n): X^T conj(X) = conj(X^dag X) has the nonzero
// spectrum of C_A.  The eigen-solver needs M to about 1e-12 absolute (the
// -lambda ln lambda of thousands of eigenvalues near 0 and 1 add up), which a
// float or split-fp16 product cannot give, so the products are made exact:
//
// Error-free splitting (the scheme of Ozaki, Ogita, Oishi and Rump, Numer.
// Algorithms 59, 2012).  Each row r of the real block Z = [Re Y | Im Y] is
// scaled by 2^-e_r, e_r the exponent bound of the row's largest entry, and
// cut into five signed 7-bit digits, toward zero:
//     Z_r = 2^e_r sum_{s<5} 2^-7(s+1) D_s[r],   D_s integers in [-127, 127]
// (exact in fp16).  The digits keep 35 bits below the row maximum: every
// float entry within a factor 2^11 of it exactly, smaller ones cut at
// 2^-35 of the maximum.  M is then the exact Gram of a matrix that close to
// Y -- Hermitian and positive semidefinite, its eigenvalues near 1 lowered by
// at most ~1e-10.
//
// The digit products D_s D_t^T are integers.  The pairs of one weight class
// c = s + t (at most five pairs) share one fp32 TMEM accumulator, which stays
// exact while it holds at most 2^24 / 127^2 = 1040 products, so it is drained
// every 3 K-blocks (5 x 192 = 960 products) into 64-bit integers:
//     H  = A_0 2^14 + A_1 2^7 + A_2,   Lo = A_3 2^21 + A_4 2^14 + A_5 2^7 + A_6,
//     M_ij = 2^(e_i + e_j - 28) H + 2^(e_i + e_j - 56) Lo     (A_c: class sums).
// Classes 7 and 8 (relative weight <= 2^-49) are left out.
//
// Re M = Z Z^T and -Im M = Z Z'^T with Z' the rows read at K + Kp mod 2 Kp and
// negated past the wrap (the same shifted operand as the state's Gram).  Only
// the lower triangle of M is written (the eigen-solver reads no more).
//
// Kernel shape: persistent CTAs, 128 x 32 output tiles of the lower triangle,
// 64-deep K-blocks of the 5 A and 5 B digit planes staged by TMA (100 KB per
// stage, two stages), 22 digit products per 16-deep K-step issued by one
// thread, two TMEM accumulator sets of 7 x 32 columns (the drain of one chunk
// overlaps the products of the next), 4 epilogue warps.  Every wait is bounded.
#include <cudaTypedefs.h>

#include <math.h>

#include <algorithm>
#include <mutex>

#include "fm_testing.h"
#include "gemm_tc.h"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace fm {
namespace xg {

using namespace ptx;

constexpr int BM = 128, BN = 32, BK = 64;
constexpr int NSLICE = 5, NCLASS = 7, CHUNK = 3, STAGES = 2;
constexpr uint32_t A_BYTES = BM * BK * 2;                       // 16 KB per digit plane
constexpr uint32_t B_BYTES = BN * BK * 2;                       // 4 KB per digit plane
constexpr uint32_t STAGE_BYTES = NSLICE * (A_BYTES + B_BYTES);  // 100 KB
constexpr uint32_t SET_COLS = NCLASS * BN;                      // one accumulator set
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
static_assert(2 * SET_COLS <= TMEM_COLS, "two accumulator sets");
static_assert(5 * 16129 * CHUNK * BK <= (1 << 24), "class sums of one chunk are exact in fp32");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");

struct GParams {
  int m;          // order of M
  int per_part;   // lower-triangle tiles of one part (Re or Im)
  int ntiles;     // 2 * per_part
  int kblocks;    // 2 Kp / BK
  int kp;         // padded contraction length Kp (multiple of BK)
  const int* expo;
  z64* M;         // m x m, column-major
  int* status;
};

// tile t -> (row tile mt, column tile nt, part); row tile mt holds the 4 (mt + 1)
// column tiles that reach its diagonal block, so 2 mt (mt + 1) tiles precede it.
FM_DEVFN void decode(int t, int per_part, int& mt, int& nt, int& part) {
  part = t >= per_part ? 1 : 0;
  t -= part * per_part;
  int a = (int)((sqrt(2.0 * t + 1.0) - 1.0) * 0.5);
  while (2 * (a + 1) * (a + 2) <= t) ++a;
  while (a > 0 && 2 * a * (a + 1) > t) --a;
  mt = a;
  nt = t - 2 * a * (a + 1);
}

// digit pairs (s, t) with s + t <= 6, grouped by class c = s + t; the first
// pair of each class starts its accumulator in a chunk
constexpr int NPAIR = 22;
FM_DEVFN void pair_of(int q, int& s, int& t, bool& first) {
  constexpr int S[NPAIR] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3, 0, 1, 2, 3, 4, 1, 2, 3, 4, 2, 3, 4};
  constexpr int T[NPAIR] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0, 4, 3, 2, 1, 0, 4, 3, 2, 1, 4, 3, 2};
  constexpr bool F[NPAIR] = {1, 1, 0, 1, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0};
  s = S[q];
  t = T[q];
  first = F[q];
}

__global__ void __launch_bounds__(256, 1)
    exact_gram_kernel(const __grid_constant__ CUtensorMap a0, const __grid_constant__ CUtensorMap a1,
                      const __grid_constant__ CUtensorMap a2, const __grid_constant__ CUtensorMap a3,
                      const __grid_constant__ CUtensorMap a4, const __grid_constant__ CUtensorMap b0,
                      const __grid_constant__ CUtensorMap b1, const __grid_constant__ CUtensorMap b2,
                      const __grid_constant__ CUtensorMap b3, const __grid_constant__ CUtensorMap b4,
                      const GParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tmem_full = empty + STAGES;   // [2]
  uint64_t* tmem_empty = tmem_full + 2;   // [2]
  uint64_t* mma_done = tmem_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tmem_full[i], 1);
      mbar_init(&tmem_empty[i], 4);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&a0); prefetch_tmap(&a1); prefetch_tmap(&a2); prefetch_tmap(&a3); prefetch_tmap(&a4);
    prefetch_tmap(&b0); prefetch_tmap(&b1); prefetch_tmap(&b2); prefetch_tmap(&b3); prefetch_tmap(&b4);
  }
  if (warp == 2) {
    tmem_alloc(tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- TMA producer
      const CUtensorMap* am[NSLICE] = {&a0, &a1, &a2, &a3, &a4};
      const CUtensorMap* bm[NSLICE] = {&b0, &b1, &b2, &b3, &b4};
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, last_phase = 0;
      for (int t = blockIdx.x; t < p.ntiles && !*abort_flag; t += gridDim.x) {
        int mt, nt, part;
        decode(t, p.per_part, mt, nt, part);
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
          const int kx = kb * BK;
          int kxb = kx;
          if (part) {
            kxb = kx + p.kp;
            if (kxb >= 2 * p.kp) kxb -= 2 * p.kp;
          }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          uint8_t* sb = sa + NSLICE * A_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
#pragma unroll
          for (int s = 0; s < NSLICE; ++s) {
            tma_load_2d(sa + s * A_BYTES, am[s], &full[stage], kx, mt * BM);
            tma_load_2d(sb + s * B_BYTES, bm[s], &full[stage], kxb, nt * BN);
          }
          issued_mask |= 1u << stage;
          if (phase) last_phase |= 1u << stage; else last_phase &= ~(1u << stage);
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      volatile int no_abort = 0;
      for (int s = 0; s < STAGES; ++s)
        if (issued_mask & (1u << s)) mbar_wait(&full[s], (last_phase >> s) & 1u, &no_abort);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------------------------------------------------------- MMA issuer
      const uint32_t id_pos = idesc_f16(BM, BN, false);
      const uint32_t id_neg = idesc_f16(BM, BN, true);
      int stage = 0;
      uint32_t phase = 0, cbuf = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
        int mt, nt, part;
        decode(t, p.per_part, mt, nt, part);
        for (int k0 = 0; k0 < p.kblocks && ok; k0 += CHUNK, ++cbuf) {
          const int k1 = min(p.kblocks, k0 + CHUNK);
          const int buf = (int)(cbuf & 1u);
          const uint32_t bpar = (cbuf >> 1) & 1u;
          if (!mbar_wait(&tmem_empty[buf], bpar ^ 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)buf * SET_COLS;
          for (int kb = k0; kb < k1; ++kb) {
            if (!mbar_wait(&full[stage], phase, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t id = (part && kb * BK >= p.kp) ? id_neg : id_pos;
            const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
            const uint32_t sb = sa + NSLICE * A_BYTES;
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) {
              const uint32_t off = j * 32;
#pragma unroll
              for (int q = 0; q < NPAIR; ++q) {
                int ps, pt;
                bool first;
                pair_of(q, ps, pt, first);
                const uint64_t da = desc_k_sw128(sa + ps * A_BYTES + off);
                const uint64_t db = desc_k_sw128(sb + pt * B_BYTES + off);
                const uint32_t accumulate = (kb > k0 || j > 0 || !first) ? 1u : 0u;
                mma_f16(acc + (uint32_t)((ps + pt) * BN), da, db, id, accumulate);
              }
            }
            mma_commit(&empty[stage]);
            if (++stage == STAGES) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&tmem_full[buf]);
        }
      }
      mma_commit(mma_done);
      volatile int no_abort = 0;
      mbar_wait(mma_done, 0, &no_abort);
    }
  } else if (warp >= 4) {
    // ---------------------------------------------------------------- epilogue
    const int ew = warp - 4;
    const int r = ew * 32 + lane;
    uint32_t cbuf = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
      int mt, nt, part;
      decode(t, p.per_part, mt, nt, part);
      long long H[BN], Lo[BN];
#pragma unroll
      for (int j = 0; j < BN; ++j) { H[j] = 0; Lo[j] = 0; }
      for (int k0 = 0; k0 < p.kblocks; k0 += CHUNK, ++cbuf) {
        const int buf = (int)(cbuf & 1u);
        const uint32_t bpar = (cbuf >> 1) & 1u;
        if (!mbar_wait(&tmem_full[buf], bpar, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t tl = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)buf * SET_COLS;
#pragma unroll
        for (int c = 0; c < NCLASS; ++c) {
          uint32_t a[32];
          tmem_ld32(tl + (uint32_t)(c * BN), a);
          tmem_wait_ld();
          const int sh = (c < 3) ? 14 - 7 * c : 21 - 7 * (c - 3);
#pragma unroll
          for (int j = 0; j < BN; ++j) {
            const long long v = (long long)__float2int_rn(__uint_as_float(a[j])) << sh;
            if (c < 3) H[j] += v;
            else Lo[j] += v;
          }
        }
        tc_fence_before();
        if (lane == 0) mbar_arrive(&tmem_empty[buf]);
      }
      if (!ok) break;
      const int i = mt * BM + r;
      if (i < p.m) {
        const int ei = p.expo[i];
#pragma unroll
        for (int j = 0; j < BN; ++j) {
          const int jj = nt * BN + j;
          if (jj <= i) {
            const int e = ei + p.expo[jj];
            const double v = scalbn((double)H[j], e - 28) + scalbn((double)Lo[j], e - 56);
            double* dst = &p.M[(int64_t)i + (int64_t)jj * p.m].re;
            dst[part] = part ? -v : v;
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag && p.status) atomicOr(p.status, FM_DEVERR_TIMEOUT);
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ------------------------------------------------------------------ digit planes
// Y[r][k] of the two layouts: ROWS_ARE_SITES (n <= N): Y = X, X[r + k ld];
// otherwise Y = X^T: X[k + r ld].  X is the n x N column-major block (leading
// dimension ld >= n) of complex128 or complex64 entries.

// rowmax[r] = max_k max(|Re Y_rk|, |Im Y_rk|) as the bits of a nonnegative double
template <typename T>
__global__ void rowmax_sites_kernel(const cplx<T>* __restrict__ X, int64_t ld, int n, int N,
                                    unsigned long long* rowmax) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int per = FM_CEIL_DIV(N, (int)gridDim.y);
  const int k0 = blockIdx.y * per, k1 = min(N, k0 + per);
  double mx = 0.0;
  for (int k = k0; k < k1; ++k) {
    const cplx<T> v = X[r + (int64_t)k * ld];
    mx = fmax(mx, fmax(fabs((double)v.re), fabs((double)v.im)));
  }
  atomicMax(&rowmax[r], (unsigned long long)__double_as_longlong(mx));
}

template <typename T>
__global__ void rowmax_orbitals_kernel(const cplx<T>* __restrict__ X, int64_t ld, int n,
                                       unsigned long long* rowmax) {
  const int r = blockIdx.x;
  double mx = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const cplx<T> v = X[k + (int64_t)r * ld];
    mx = fmax(mx, fmax(fabs((double)v.re), fabs((double)v.im)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    rowmax[r] = (unsigned long long)__double_as_longlong(fmax(mx, red[0]));
  }
}

// e_r with max_k |Z_rk| < 2^e_r (0 for a zero or padding row)
__global__ void exponents_kernel(const unsigned long long* rowmax, int m, int mp, int* expo) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mp) return;
  const double mx = r < m ? __longlong_as_double((long long)rowmax[r]) : 0.0;
  expo[r] = mx > 0.0 ? ilogb(mx) + 1 : 0;
}

// the NSLICE signed 7-bit digits of v 2^-e (|v| < 2^e), toward zero; exact steps in float64
FM_DEVFN void digits(double v, int e, __half (&d)[NSLICE]) {
  double x = scalbn(v, 7 - e);
#pragma unroll
  for (int s = 0; s < NSLICE; ++s) {
    const double q = trunc(x);
    d[s] = __float2half_rn((float)q);   // |q| <= 127: exact
    x = (x - q) * 128.0;
  }
}

// planes[s][r][kk], kk < Kp: Re Y[r][kk], kk >= Kp: Im Y[r][kk - Kp]; zero padding
// outside m x Kc.  32 x 32 tiles through shared memory so that both the read of
// X and the write of the planes are coalesced.
template <bool ROWS_ARE_SITES, typename T>
__global__ void slice_kernel(const cplx<T>* __restrict__ X, int64_t ld, int m, int Kc, int Kp,
                             const int* __restrict__ expo, __half* planes, int64_t plane_stride) {
  __shared__ z64 tile[32][33];   // [k][r]
  const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = ty + 8 * q;
    z64 v = cmk(0.0, 0.0);
    if (ROWS_ARE_SITES) {       // read along r
      const int r = r0 + tx, k = k0 + a;
      if (r < m && k < Kc) {
        const cplx<T> x = X[r + (int64_t)k * ld];
        v = cmk((double)x.re, (double)x.im);
      }
      tile[a][tx] = v;
    } else {                    // read along k
      const int k = k0 + tx, r = r0 + a;
      if (r < m && k < Kc) {
        const cplx<T> x = X[k + (int64_t)r * ld];
        v = cmk((double)x.re, (double)x.im);
      }
      tile[tx][a] = v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int rl = ty + 8 * q;
    const int r = r0 + rl, k = k0 + tx;
    const z64 v = tile[tx][rl];
    const int e = expo[r];
    __half dr[NSLICE], di[NSLICE];
    digits(v.re, e, dr);
    digits(v.im, e, di);
    const int64_t o = (int64_t)r * 2 * Kp + k;
#pragma unroll
    for (int s = 0; s < NSLICE; ++s) {
      planes[s * plane_stride + o] = dr[s];
      planes[s * plane_stride + o + Kp] = di[s];
    }
  }
}

}  // namespace xg

namespace {
struct XgLayout {
  int m, Kc, mp, Kp;
  size_t planes_bytes, rowmax_off, expo_off, total;
};
XgLayout xg_layout(int n, int N) {
  XgLayout l;
  const bool sites = n <= N;
  l.m = sites ? n : N;
  l.Kc = sites ? N : n;
  l.mp = FM_CEIL_DIV(l.m, xg::BM) * xg::BM;
  l.Kp = FM_CEIL_DIV(l.Kc, xg::BK) * xg::BK;
  l.planes_bytes = (size_t)xg::NSLICE * l.mp * 2 * l.Kp * 2;
  l.rowmax_off = (l.planes_bytes + 255) & ~(size_t)255;
  l.expo_off = l.rowmax_off + (((size_t)l.mp * 8 + 255) & ~(size_t)255);
  l.total = l.expo_off + (((size_t)l.mp * 4 + 255) & ~(size_t)255);
  return l;
}
}  // namespace

// scratch of exact_gram for every subsystem size n <= nmax (the two layouts peak at n = N and n = nmax)
size_t exact_gram_scratch_bytes(int nmax, int N) {
  size_t b = xg_layout(std::min(nmax, N), N).total;
  if (nmax > N) b = std::max(b, xg_layout(nmax, N).total);
  return b;
}

template <typename T>
cudaError_t exact_gram_t(cudaStream_t st, const cplx<T>* X, int64_t ld, int n, int N, z64* M, void* scratch,
                         int* status, int64_t* launches) {
  using namespace xg;
  const bool sites = n <= N;
  const XgLayout l = xg_layout(n, N);
  const int m = l.m, Kc = l.Kc, mp = l.mp, Kp = l.Kp;
  if (m <= 0) return cudaSuccess;
  const int64_t plane_stride = (int64_t)mp * 2 * Kp;
  char* base = (char*)scratch;
  __half* planes = (__half*)base;
  unsigned long long* rowmax = (unsigned long long*)(base + l.rowmax_off);
  int* expo = (int*)(base + l.expo_off);
  cudaError_t e;
  if ((e = cudaMemsetAsync(rowmax, 0, (size_t)mp * 8, st))) return e;
  if (sites) {
    const int gy = std::max(1, std::min(64, (4 * 152) / std::max(1, FM_CEIL_DIV(m, 256))));
    rowmax_sites_kernel<T><<<dim3(FM_CEIL_DIV(m, 256), gy), 256, 0, st>>>(X, ld, n, N, rowmax);
  } else {
    rowmax_orbitals_kernel<T><<<m, 256, 0, st>>>(X, ld, n, rowmax);
  }
  exponents_kernel<<<FM_CEIL_DIV(mp, 256), 256, 0, st>>>(rowmax, m, mp, expo);
  const dim3 sg(Kp / 32, mp / 32), sb(32, 8);
  if (sites) slice_kernel<true, T><<<sg, sb, 0, st>>>(X, ld, m, Kc, Kp, expo, planes, plane_stride);
  else slice_kernel<false, T><<<sg, sb, 0, st>>>(X, ld, m, Kc, Kp, expo, planes, plane_stride);
  if ((e = cudaGetLastError())) return e;
  CUtensorMap am[NSLICE], bm[NSLICE];
  for (int s = 0; s < NSLICE; ++s) {
    const __half* pl = planes + s * plane_stride;
    if (!tc::make_kmajor_map(&am[s], pl, 2 * (uint64_t)Kp, mp, 2 * (uint64_t)Kp, BM) ||
        !tc::make_kmajor_map(&bm[s], pl, 2 * (uint64_t)Kp, mp, 2 * (uint64_t)Kp, BN))
      return cudaErrorInvalidValue;
  }
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(exact_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  });
  if (attr != cudaSuccess) return attr;
  GParams p;
  p.m = m;
  const int mtiles = mp / BM;
  p.per_part = 2 * mtiles * (mtiles + 1);
  p.ntiles = 2 * p.per_part;
  p.kblocks = 2 * Kp / BK;
  p.kp = Kp;
  p.expo = expo;
  p.M = M;
  p.status = status;
  const int grid = std::min(p.ntiles, tc::sm_count());
  exact_gram_kernel<<<grid, 256, SMEM_BYTES, st>>>(am[0], am[1], am[2], am[3], am[4], bm[0], bm[1], bm[2], bm[3],
                                                   bm[4], p);
  if ((e = cudaGetLastError())) return e;
  if (launches) *launches += 5;
  return cudaSuccess;
}

cudaError_t exact_gram(cudaStream_t st, const z64* X, int n, int N, z64* M, void* scratch, int* status,
                       int64_t* launches) {
  return exact_gram_t<double>(st, X, n, n, N, M, scratch, status, launches);
}

cudaError_t exact_gram_c32(cudaStream_t st, const c32* X, int64_t ld, int n, int N, z64* M, void* scratch,
                           int* status, int64_t* launches) {
  return exact_gram_t<float>(st, X, ld, n, N, M, scratch, status, launches);
}

}  // namespace fm

// ====================================================================== projector correction
// The float state is orthonormal only to ~1e-7 (G = U^dag U = 1 + E), and C = U U^dag
// is then not a projector: its eigenvalues near 1 sit ~|E| off 1, and -d ln d over
// thousands of them biases the entropy by ~1e-3 at l = 8192.  The state's C is the
// projector onto span(U), U G^-1 U^dag; to first order in E (|E|^2 ~ 1e-14):
//   n <= N:  C_A = U_A G^-1 U_A^dag      ~ M - U_A E U_A^dag
//   n >  N:  spectrum of G^-1/2 U_A^dag U_A G^-1/2 ~ M_t - (E M_t + M_t E) / 2,
//            M = conj(M_t)  ->  M - (conj(E) M + M conj(E)) / 2.
// The products carry the factor E, so complex64 products leave errors ~1e-14; the
// subtraction is done in float64 on the lower triangle.
namespace fm {
namespace xg {

// Ec = (conj ? conj(Gx) : Gx) - 1 as complex64, full from the lower triangle of Gx (m x m)
__global__ void e_from_gram_kernel(const z64* __restrict__ Gx, int m, int conj_, c32* Ec) {
  const int64_t tot = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    z64 g = i >= j ? Gx[i + (int64_t)j * m] : cconj(Gx[j + (int64_t)i * m]);
    if (conj_) g = cconj(g);
    if (i == j) g.re -= 1.0;
    Ec[idx] = cmk((float)g.re, (float)g.im);
  }
}

// complex64 copy of a complex128 array; herm != 0: m x m Hermitian, full from the lower triangle
__global__ void to_c32_kernel(const z64* __restrict__ X, int64_t n, int m, int herm, c32* Y) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n; idx += (int64_t)gridDim.x * blockDim.x) {
    z64 v;
    if (herm) {
      const int i = (int)(idx % m), j = (int)(idx / m);
      v = i >= j ? X[i + (int64_t)j * m] : cconj(X[j + (int64_t)i * m]);
    } else {
      v = X[idx];
    }
    Y[idx] = cmk((float)v.re, (float)v.im);
  }
}

// lower triangle of M -= D (sym == 0) or M -= (Z + Z^dag) / 2 (sym != 0), D / Z complex64 m x m
__global__ void sub_lower_kernel(z64* M, int m, const c32* __restrict__ D, int sym) {
  const int64_t tot = (int64_t)m * m;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot; idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx % m), j = (int)(idx / m);
    if (i < j) continue;
    double dr = D[idx].re, di = D[idx].im;
    if (sym) {
      const c32 t = D[j + (int64_t)i * m];
      dr = 0.5 * (dr + (double)t.re);
      di = 0.5 * (di - (double)t.im);
    }
    M[idx].re -= dr;
    M[idx].im -= di;
  }
}

}  // namespace xg

size_t projector_scratch_bytes(int N) { return (size_t)4 * N * N * sizeof(c32) + 1024; }

cudaError_t projector_correct(cudaStream_t st, const z64* Gx, const z64* XA, int n, int N, z64* M, void* scratch,
                              int64_t* launches) {
  using namespace xg;
  const int m = std::min(n, N);
  const bool sites = n <= N;
  c32* Ec = (c32*)scratch;                       // N x N
  c32* A = Ec + (int64_t)N * N;                  // n <= N: U_A (n x N); else M as complex64 (N x N)
  c32* P = A + (int64_t)N * N;                   // products
  c32* D = P + (int64_t)N * N;
  const c32 one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
  e_from_gram_kernel<<<152 * 8, 256, 0, st>>>(Gx, N, sites ? 1 : 0, Ec);
  cudaError_t e;
  if (sites) {
    to_c32_kernel<<<152 * 8, 256, 0, st>>>(XA, (int64_t)n * N, n, 0, A);
    if ((e = zgemm<float>(st, n, N, N, OP_N, OP_N, one, A, n, 0, Ec, N, 0, zero, P, n, 0, 1, 0))) return e;
    if ((e = zgemm<float>(st, n, n, N, OP_N, OP_C, one, P, n, 0, A, n, 0, zero, D, n, 0, 1, GEMM_LOWER_ONLY)))
      return e;
    sub_lower_kernel<<<152 * 8, 256, 0, st>>>(M, m, D, 0);
  } else {
    to_c32_kernel<<<152 * 8, 256, 0, st>>>(M, (int64_t)N * N, N, 1, A);
    if ((e = zgemm<float>(st, N, N, N, OP_N, OP_N, one, Ec, N, 0, A, N, 0, zero, D, N, 0, 1, 0))) return e;
    sub_lower_kernel<<<152 * 8, 256, 0, st>>>(M, m, D, 1);
  }
  if (launches) *launches += 5;
  return cudaGetLastError();
}

}  // namespace fm

// ====================================================================== test hooks
extern "C" unsigned long long fmx_exact_gram_scratch_bytes(int nmax, int N) {
  return (unsigned long long)fm::exact_gram_scratch_bytes(nmax, N);
}

extern "C" int fmx_exact_gram(const void* X, int n, int N, void* M, void* d_scratch, void* stream) {
  if (n < 1 || N < 1) return (int)cudaErrorInvalidValue;
  return (int)fm::exact_gram((cudaStream_t)stream, (const z64*)X, n, N, (z64*)M, d_scratch, nullptr,
                             nullptr);
}
