// Split-fp16 tensor-core GEMM for sm_103a (tcgen05 + TMEM + TMA).
//
// D[m, n] = sum_k A[m, k] B[n, k] with both operands K-major and each given as
// two fp16 planes, x = h + l * 2^-11 (|x - h - l 2^-11| <~ 2^-22 |x|).  Three
// tensor-core products per K-step, accumulated in fp32 in TMEM:
//   acc0 += Ah Bh,   acc1 += Ah Bl + Al Bh,   D = acc0 + 2^-11 acc1.
// The dropped Al Bl term is ~2^-22 relative.
//
// Kernel shape: persistent CTAs (one per SM), 128 x BN output tiles, K-blocks
// of 64 (one 128-byte swizzle row), STAGES-deep TMA -> shared memory pipeline.
// Warp 0 issues TMA, warp 1 issues MMAs (one thread), warp 2 owns TMEM,
// warps 4-7 drain TMEM into the mode's epilogue.  Every wait is bounded and
// raises FM_DEVERR_TIMEOUT instead of hanging.
#include <atomic>
#include <cstring>
#include <mutex>
#include <cudaTypedefs.h>

#include <vector>

#include "gemm_tc.h"
#include "tc_ptx.cuh"

namespace fm {
namespace tc {

using namespace ptx;

template <int BN, int CHUNKED>
struct Cfg {
  static constexpr int STAGES = (BN == 256) ? 2 : 3;
  static constexpr uint32_t A_BYTES = BM * BK * 2;
  static constexpr uint32_t B_BYTES = BN * BK * 2;
  static constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  // TMEM accumulator sets: two (the epilogue of one tile or chunk overlaps the
  // MMAs of the next) whenever both fit in the 512 columns
  static constexpr int NBUF = (CHUNKED || BN <= 128) ? 2 : 1;
  static constexpr uint32_t TMEM_COLS = (NBUF * 2 * BN <= 256) ? 256 : 512;
  static constexpr uint32_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static_assert(NBUF * 2 * BN <= 512, "TMEM holds 512 columns");
};

struct TileInfo {
  int mt, nt, b, part;
};

// The tile at position t of the persistent loop of a launch of G CTAs (CTA i takes the
// positions i, i + G, ...); host and device (the host side serves fmx_tile_order).
__host__ __device__ __forceinline__ TileInfo decode_order(const Params& p, int t, int G) {
  TileInfo ti;
  if (p.order == ORDER_PAIRS_A || p.order == ORDER_PAIRS_B) {
    // units = pairs of tiles; rounds 2k and 2k + 1 of the persistent loop take the two
    // members of the same G units in the same CTA order (the last, partial round pair:
    // its members side by side)
    const int U = p.ntiles >> 1;
    const int kp = t / (2 * G), full = U / G, rem = U - full * G;
    const int rr = t - kp * 2 * G;
    const int which = kp < full ? rr / G : rr / rem;
    const int u = kp * G + (kp < full ? rr - which * G : rr - which * rem);
    const int M = p.mt_mod;
    if (p.order == ORDER_PAIRS_A) {
      const int P2 = M >> 1, pr = u % P2;
      int rest = u / P2;
      ti.nt = rest % p.ntiles_n;
      rest /= p.ntiles_n;
      const bool high = (which == 0) == (p.kb_hi_mt != 0);   // the heavier member first
      ti.mt = (rest & 1) * M + (high ? M - 1 - pr : pr);
      ti.b = rest >> 1;
    } else {
      const int P2 = p.ntiles_n >> 1, pn = u % P2;
      const int rest = u / P2;
      ti.mt = rest % p.mtiles;
      ti.b = rest / p.mtiles;
      ti.nt = which == 0 ? p.ntiles_n - 1 - pn : pn;
    }
    ti.part = 0;
    return ti;
  }
  if (p.order == ORDER_HERM) {
    // the upper tiles of each (batch item, Re / Im half): groups of 16 row tiles, each
    // sweeping its columns nt >= its first row (column j of a group holds min(16, j + 1) rows)
    const int M = p.mt_mod, T = M * (M + 1) / 2;
    const int bp = t / T;
    int r = t - bp * T, g0 = 0;
    for (;;) {
      const int w = M - g0;
      const int size = w <= 16 ? w * (w + 1) / 2 : 136 + (w - 16) * 16;
      if (r < size) break;
      r -= size;
      g0 += 16;
    }
    int j, ro;
    if (r < 136 || M - g0 <= 16) {
      j = 0;
      while ((j + 1) * (j + 2) / 2 <= r) ++j;
      ro = r - j * (j + 1) / 2;
    } else {
      j = 16 + (r - 136) / 16;
      ro = (r - 136) % 16;
    }
    ti.mt = (bp & 1) * M + g0 + ro;
    ti.nt = g0 + j;
    ti.b = bp >> 1;
    ti.part = 0;
    return ti;
  }
  // grouped raster: 16 consecutive m-tiles sweep all n-tiles
  const int per_b = p.mtiles * p.ntiles_n;
  ti.b = t / per_b;
  t -= ti.b * per_b;
  const int GM = 16;
  const int group = t / (GM * p.ntiles_n);
  const int first_m = group * GM;
  const int gsz = p.mtiles - first_m < GM ? p.mtiles - first_m : GM;
  const int r = t - group * GM * p.ntiles_n;
  ti.mt = first_m + r % gsz;
  ti.nt = r / gsz;
  ti.part = 0;
  return ti;
}

__device__ __forceinline__ TileInfo decode(const Params& p, int t) {
  if (p.tiles) {
    const int4 v = p.tiles[t];
    TileInfo ti;
    ti.mt = v.x; ti.nt = v.y; ti.b = v.z; ti.part = v.w;
    return ti;
  }
  return decode_order(p, t, gridDim.x);
}

// One 32-column slab of a finished tile: row r of the tile, columns c0..c0+31.
template <int BN, int MODE>
__device__ __forceinline__ void emit(const Params& p, const TileInfo& ti, int r, int c0, const float (&d)[32],
                                     double& rowsum) {
  const int m0 = ti.mt * BM, n0 = ti.nt * BN;
  if (MODE == MODE_PLAIN) {
    float* out = p.out_f + (int64_t)ti.b * p.out_batch_stride + (int64_t)(m0 + r) + (int64_t)(n0 + c0) * p.ld_out;
#pragma unroll
    for (int j = 0; j < 32; ++j) out[(int64_t)j * p.ld_out] = d[j];
  } else if (MODE == MODE_PROP) {
    // row sums of squares: float over the slab's 32 columns (fixed order), then one double add
    float* out = p.out_f + (int64_t)(m0 + r) + (int64_t)(n0 + c0) * p.ld_out;
    float part = 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      out[(int64_t)j * p.ld_out] = d[j];
      part = fmaf(d[j], d[j], part);
    }
    rowsum += (double)part;
  } else if (MODE == MODE_GRAM) {
    // complex64 G_b[k1 + k2 N], real or imaginary part
    float* out = p.out_gf + 2 * ((int64_t)ti.b * p.Ntraj * p.Ntraj + (int64_t)(m0 + r) +
                                 (int64_t)(n0 + c0) * p.Ntraj) + ti.part;
#pragma unroll
    for (int j = 0; j < 32; ++j) out[2 * (int64_t)j * p.Ntraj] = d[j];
    if (p.estat) {
      // largest off-diagonal |entry| of this row's slab (rowsum carries the running max)
      float mx = (float)rowsum;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (m0 + r != n0 + c0 + j) mx = fmaxf(mx, fabsf(d[j]));
      rowsum = (double)mx;
    }
  } else if (MODE == MODE_ADDV) {
    // all 32 loads before the first store: the stores could alias the loads as far as
    // the compiler knows, so interleaving them would serialise on memory latency
    const int64_t o0 = (int64_t)ti.b * p.out_batch_stride + (int64_t)(m0 + r) + (int64_t)(n0 + c0) * p.ld_out;
    float x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = __ldg(&p.in_f[o0 + (int64_t)j * p.ld_out]);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t o = o0 + (int64_t)j * p.ld_out;
      const float v = x[j] + d[j];
      p.out_f[o] = v;
      const __half h = __float2half_rn(v);
      p.out_h[o] = h;
      p.out_l[o] = __float2half_rn((v - __half2float(h)) * 2048.0f);
    }
  } else if (MODE == MODE_CPLX) {
    // row tile mt < mt_mod: real parts of rows mt BM .. ; mt >= mt_mod: imaginary parts
    const int part = ti.mt >= p.mt_mod ? 1 : 0;
    const int64_t row = (int64_t)(ti.mt - part * p.mt_mod) * BM + r;
    float* out = p.out_c + 2 * ((int64_t)ti.b * p.out_batch_stride + row + (int64_t)(n0 + c0) * p.ld_out) + part;
    if (p.beta != 0.0f) {
      float x[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x[j] = out[2 * (int64_t)j * p.ld_out];
#pragma unroll
      for (int j = 0; j < 32; ++j) out[2 * (int64_t)j * p.ld_out] = p.alpha * d[j] + p.beta * x[j];
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) out[2 * (int64_t)j * p.ld_out] = p.alpha * d[j];
    }
  } else {  // MODE_TRMM: column c of the L x 2N view -> V_b[(c&1) L + i + (c>>1) 2L]
    const int64_t base = (int64_t)ti.b * 2 * p.L * p.Ntraj + (m0 + r);
    float x[32];                              // loads first (see MODE_ADDV)
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = n0 + c0 + j;
      x[j] = p.in_f ? __ldg(&p.in_f[base + (int64_t)(c & 1) * p.L + (int64_t)(c >> 1) * 2 * p.L]) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = n0 + c0 + j;
      const int64_t o = base + (int64_t)(c & 1) * p.L + (int64_t)(c >> 1) * 2 * p.L;
      const float v = x[j] + d[j];
      p.out_f[o] = v;
      const __half h = __float2half_rn(v);
      p.out_h[o] = h;
      p.out_l[o] = __float2half_rn((v - __half2float(h)) * 2048.0f);
    }
  }
}

// K-blocks [x, y) of a tile; the host guarantees x < y for every tile that is not skipped.
template <int BN>
__device__ __forceinline__ int2 krange(const Params& p, const TileInfo& ti) {
  int lo = 0, hi = p.kblocks;
  if (p.tri_k) hi = min(hi, (ti.nt + 1) * BN / BK);
  const int mr = p.mt_mod > 0 ? ti.mt % p.mt_mod : ti.mt;
  if (p.kb_lo_mt) lo = mr * p.kb_lo_mt;
  if (p.kb_hi_mt) hi = min(hi, (mr + 1) * p.kb_hi_mt);
  if (p.kb_hi_nt) hi = min(hi, (ti.nt + 1) * p.kb_hi_nt);
  return make_int2(lo, hi);
}

__device__ __forceinline__ bool tile_skipped(const Params& p, const TileInfo& ti) {
  return p.herm_upper && ti.mt % p.mt_mod > ti.nt;
}

template <int BN, int CHUNKED, int MODE>
__global__ void __launch_bounds__(256, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                   const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                   const Params p) {
  using C = Cfg<BN, CHUNKED>;
  if (p.cond && *(volatile const int*)p.cond == 0) return;   // uniform: before any barrier or TMEM
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* tmem_full = empty + C::STAGES;       // [NBUF]
  uint64_t* tmem_empty = tmem_full + 2;          // [NBUF]
  uint64_t* mma_done = tmem_empty + 2;
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int i = 0; i < C::NBUF; ++i) {
      mbar_init(&tmem_full[i], 1);
      mbar_init(&tmem_empty[i], 4);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    fence_mbar_init();
    prefetch_tmap(&tmAh); prefetch_tmap(&tmAl); prefetch_tmap(&tmBh); prefetch_tmap(&tmBl);
  }
  if (warp == 2) {
    tmem_alloc(tmem_slot, C::TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------------------------------------------------------- TMA producer
      int stage = 0;
      uint32_t phase = 0;
      uint32_t issued_mask = 0, last_phase = 0;
      for (int t = blockIdx.x; t < p.ntiles && !*abort_flag; t += gridDim.x) {
        const TileInfo ti = decode(p, t);
        if (tile_skipped(p, ti)) continue;
        const int2 kr = krange<BN>(p, ti);
        const int arow = ti.b * p.a_rows_per_b + ti.mt * BM;
        const int brow = ti.b * p.b_rows_per_b + ti.nt * BN;
        for (int kb = kr.x; kb < kr.y; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag)) break;
          const int kx = kb * BK;
          int kxb = kx;
          if (p.k_shift && ti.part == 1) {
            kxb = kx + p.k_shift;
            if (kxb >= p.kdim) kxb -= p.kdim;
          }
          uint8_t* sAh = smem + stage * C::STAGE_BYTES;
          uint8_t* sAl = sAh + C::A_BYTES;
          uint8_t* sBh = sAl + C::A_BYTES;
          uint8_t* sBl = sBh + C::B_BYTES;
          mbar_expect_tx(&full[stage], C::STAGE_BYTES);
          tma_load_2d(sAh, &tmAh, &full[stage], kx, arow);
          tma_load_2d(sAl, &tmAl, &full[stage], kx, arow);
          tma_load_2d(sBh, &tmBh, &full[stage], kxb, brow);
          tma_load_2d(sBl, &tmBl, &full[stage], kxb, brow);
          issued_mask |= 1u << stage;
          if (phase) last_phase |= 1u << stage; else last_phase &= ~(1u << stage);
          if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
        }
      }
      // never leave the CTA with copies still landing in its shared memory
      volatile int no_abort = 0;
      for (int s = 0; s < C::STAGES; ++s)
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
        const TileInfo ti = decode(p, t);
        if (tile_skipped(p, ti)) continue;
        const int2 kr = krange<BN>(p, ti);
        const int ckb = CHUNKED ? p.chunk_kb : kr.y - kr.x;
        for (int k0 = kr.x; k0 < kr.y && ok; k0 += ckb, ++cbuf) {
          const int k1 = min(kr.y, k0 + ckb);
          const int buf = (int)(cbuf % C::NBUF);
          const uint32_t bpar = (cbuf / C::NBUF) & 1u;
          if (!mbar_wait(&tmem_empty[buf], bpar ^ 1, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t acc0 = tmem + (uint32_t)(buf * 2 * BN), acc1 = acc0 + BN;
          for (int kb = k0; kb < k1; ++kb) {
            if (!mbar_wait(&full[stage], phase, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const bool neg = p.k_shift && ti.part == 1 && (kb * BK >= p.kdim - p.k_shift);
            const uint32_t id = neg ? id_neg : id_pos;
            const uint32_t sAh = smem_u32(smem + stage * C::STAGE_BYTES);
            const uint32_t sAl = sAh + C::A_BYTES;
            const uint32_t sBh = sAl + C::A_BYTES;
            const uint32_t sBl = sBh + C::B_BYTES;
#pragma unroll
            for (int j = 0; j < BK / 16; ++j) {
              const uint32_t off = j * 32;  // 16 fp16 = 32 bytes along K inside the swizzle row
              const uint64_t ah = desc_k_sw128(sAh + off), al = desc_k_sw128(sAl + off);
              const uint64_t bh = desc_k_sw128(sBh + off), bl = desc_k_sw128(sBl + off);
              const uint32_t acc = (kb > k0 || j > 0) ? 1u : 0u;
              mma_f16(acc0, ah, bh, id, acc);
              mma_f16(acc1, ah, bl, id, acc);
              mma_f16(acc1, al, bh, id, 1u);
            }
            mma_commit(&empty[stage]);
            if (++stage == C::STAGES) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&tmem_full[buf]);
        }
      }
      // all MMAs retired before TMEM can be released
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
      const TileInfo ti = decode(p, t);
      if (tile_skipped(p, ti)) continue;
      const int2 kr = krange<BN>(p, ti);
      double rowsum = 0.0;
      if (CHUNKED) {
        // running fp32 sums of the whole tile row, fed chunk by chunk (round to nearest)
        float S[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) S[j] = 0.0f;
        for (int k0 = kr.x; k0 < kr.y; k0 += p.chunk_kb, ++cbuf) {
          const int buf = (int)(cbuf % C::NBUF);
          const uint32_t bpar = (cbuf / C::NBUF) & 1u;
          if (!mbar_wait(&tmem_full[buf], bpar, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t tl0 = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * 2 * BN);
#pragma unroll
          for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t a0[32], a1[32];
            tmem_ld32(tl0 + c0, a0);
            tmem_ld32(tl0 + BN + c0, a1);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 32; ++j)
              S[c0 + j] += __uint_as_float(a0[j]) + __uint_as_float(a1[j]) * (1.0f / 2048.0f);
          }
          tc_fence_before();
          if (lane == 0) mbar_arrive(&tmem_empty[buf]);
        }
        if (!ok) break;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
          float d[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) d[j] = S[c0 + j];
          emit<BN, MODE>(p, ti, r, c0, d, rowsum);
        }
      } else {
        const int buf = (int)(cbuf % C::NBUF);
        const uint32_t bpar = (cbuf / C::NBUF) & 1u;
        if (!mbar_wait(&tmem_full[buf], bpar, abort_flag)) { ok = false; break; }
        tc_fence_after();
        for (int c0 = 0; c0 < BN; c0 += 32) {
          uint32_t a0[32], a1[32];
          const uint32_t tl = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * 2 * BN) + (uint32_t)c0;
          tmem_ld32(tl, a0);
          tmem_ld32(tl + BN, a1);
          tmem_wait_ld();
          float d[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) d[j] = __uint_as_float(a0[j]) + __uint_as_float(a1[j]) * (1.0f / 2048.0f);
          emit<BN, MODE>(p, ti, r, c0, d, rowsum);
        }
        tc_fence_before();
        if (lane == 0) mbar_arrive(&tmem_empty[buf]);
        ++cbuf;
      }
      if (MODE == MODE_GRAM && p.estat) {
        const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint((float)rowsum));
        if (lane == 0) atomicMax(&p.estat[2 * ti.b + 1], m);
      }
      if (MODE == MODE_PROP) {
        const int R = ti.mt * BM + r;
        const int n0 = ti.nt * BN;
        const int b = n0 / p.Ntraj, cidx = (n0 % p.Ntraj) / BN;
        p.partial[((int64_t)b * p.C + cidx) * 2 * p.L + R] = rowsum;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abort_flag && p.status) atomicOr(p.status, FM_DEVERR_TIMEOUT);
  if (warp == 2) {
    tc_fence_after();
    tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ------------------------------------------------------------------ host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

// K-major fp16 plane: `rows` rows of `K` contiguous elements, row pitch `ld` elements.
bool make_kmajor_map(CUtensorMap* m, const __half* base, uint64_t K, uint64_t rows, uint64_t ld, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t smem_bytes(int BN) { return BN == 256 ? Cfg<256, 0>::SMEM_BYTES : Cfg<128, 0>::SMEM_BYTES; }

template <int BN, int CH, int MODE>
static cudaError_t set_smem() {
  return cudaFuncSetAttribute(tc_gemm_kernel<BN, CH, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)Cfg<BN, CH>::SMEM_BYTES);
}

// Shared-memory opt-in of every instantiation, done once before any launch (so
// that no attribute call falls inside a stream capture).
cudaError_t configure_all() {
  static std::atomic<bool> done{false};
  static std::mutex mu;
  if (done.load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  if (done.load(std::memory_order_relaxed)) return cudaSuccess;
  cudaError_t e;
  if ((e = set_smem<256, 0, MODE_PLAIN>()) || (e = set_smem<128, 0, MODE_PLAIN>()) ||
      (e = set_smem<128, 1, MODE_PLAIN>()) || (e = set_smem<256, 0, MODE_PROP>()) ||
      (e = set_smem<128, 0, MODE_PROP>()) || (e = set_smem<256, 0, MODE_GRAM>()) ||
      (e = set_smem<128, 0, MODE_GRAM>()) || (e = set_smem<128, 1, MODE_TRMM>()) ||
      (e = set_smem<128, 0, MODE_TRMM>()) || (e = set_smem<256, 0, MODE_TRMM>()) ||
      (e = set_smem<128, 0, MODE_ADDV>()) || (e = set_smem<256, 0, MODE_ADDV>()) ||
      (e = set_smem<128, 0, MODE_CPLX>()))
    return e;
  done.store(true, std::memory_order_release);
  return cudaSuccess;
}

template <int BN, int CH, int MODE>
static cudaError_t launch_one(cudaStream_t st, const CUtensorMap& Ah, const CUtensorMap& Al, const CUtensorMap& Bh,
                              const CUtensorMap& Bl, const Params& p, int grid) {
  cudaError_t e = configure_all();
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<BN, CH, MODE><<<grid, 256, Cfg<BN, CH>::SMEM_BYTES, st>>>(Ah, Al, Bh, Bl, p);
  return cudaGetLastError();
}

// One kernel instantiation per (tile width, accumulation, epilogue), so each
// product of the step is a distinct kernel in profiles.
cudaError_t launch(cudaStream_t st, int BN, const CUtensorMap& Ah, const CUtensorMap& Al, const CUtensorMap& Bh,
                   const CUtensorMap& Bl, const Params& p, int grid) {
  if (p.ntiles <= 0) return cudaSuccess;
  if (grid <= 0 || grid > p.ntiles) grid = p.ntiles;
  const bool ch = p.chunk_kb > 0;
  if (ch && BN != 128) return cudaErrorInvalidValue;
  switch (p.mode) {
    case MODE_PLAIN:
      if (ch) return launch_one<128, 1, MODE_PLAIN>(st, Ah, Al, Bh, Bl, p, grid);
      return BN == 256 ? launch_one<256, 0, MODE_PLAIN>(st, Ah, Al, Bh, Bl, p, grid)
                       : launch_one<128, 0, MODE_PLAIN>(st, Ah, Al, Bh, Bl, p, grid);
    case MODE_PROP:
      if (ch) return cudaErrorInvalidValue;
      return BN == 256 ? launch_one<256, 0, MODE_PROP>(st, Ah, Al, Bh, Bl, p, grid)
                       : launch_one<128, 0, MODE_PROP>(st, Ah, Al, Bh, Bl, p, grid);
    case MODE_GRAM:
      if (ch) return cudaErrorInvalidValue;
      return BN == 256 ? launch_one<256, 0, MODE_GRAM>(st, Ah, Al, Bh, Bl, p, grid)
                       : launch_one<128, 0, MODE_GRAM>(st, Ah, Al, Bh, Bl, p, grid);
    case MODE_ADDV:
      if (ch) return cudaErrorInvalidValue;
      return BN == 256 ? launch_one<256, 0, MODE_ADDV>(st, Ah, Al, Bh, Bl, p, grid)
                       : launch_one<128, 0, MODE_ADDV>(st, Ah, Al, Bh, Bl, p, grid);
    case MODE_CPLX:
      if (ch || BN != 128) return cudaErrorInvalidValue;
      return launch_one<128, 0, MODE_CPLX>(st, Ah, Al, Bh, Bl, p, grid);
    case MODE_TRMM:
      if (ch) return launch_one<128, 1, MODE_TRMM>(st, Ah, Al, Bh, Bl, p, grid);
      return BN == 256 ? launch_one<256, 0, MODE_TRMM>(st, Ah, Al, Bh, Bl, p, grid)
                       : launch_one<128, 0, MODE_TRMM>(st, Ah, Al, Bh, Bl, p, grid);
  }
  return cudaErrorInvalidValue;
}

// Tile list in grouped order: GM consecutive m-tiles sweep all n-tiles, so the
// CTAs resident at one time share A rows and B columns in L2.
std::vector<int4> tile_list(int mtiles, int ntiles, int batch, int parts, bool upper_only, int BN, int GM) {
  std::vector<int4> out;
  for (int b = 0; b < batch; ++b)
    for (int part = 0; part < parts; ++part)
      for (int g0 = 0; g0 < mtiles; g0 += GM) {
        const int g1 = std::min(mtiles, g0 + GM);
        for (int nt = 0; nt < ntiles; ++nt)
          for (int mt = g0; mt < g1; ++mt) {
            if (upper_only && mt * BM > nt * BN + BN - 1) continue;
            out.push_back(make_int4(mt, nt, b, part));
          }
      }
  return out;
}

int sm_count() {
  static const int n = [] {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
  }();
  return n;
}

}  // namespace tc
}  // namespace fm

// Host-only test hook: the tiles of one launch in the order the persistent loop takes them.
extern "C" int fmx_tile_order(int order, int mt_mod, int ntiles_n, int batch, int lower, int grid, int* out,
                              int cap) {
  using namespace fm::tc;
  if (!out || order < ORDER_RASTER || order > ORDER_HERM || mt_mod < 1 || ntiles_n < 1 || batch < 1 || grid < 1 ||
      (order == ORDER_PAIRS_A && mt_mod % 2) || (order == ORDER_PAIRS_B && ntiles_n % 2) ||
      (order == ORDER_HERM && ntiles_n != mt_mod))
    return -1;
  Params p;
  memset(&p, 0, sizeof(p));
  p.order = order;
  p.mt_mod = mt_mod;
  p.mtiles = 2 * mt_mod;
  p.ntiles_n = ntiles_n;
  p.kb_hi_mt = lower ? 4 : 0;
  p.kb_lo_mt = lower ? 0 : 4;
  const int64_t n = order == ORDER_HERM ? (int64_t)batch * mt_mod * (mt_mod + 1) : (int64_t)batch * 2 * mt_mod * ntiles_n;
  if (n > cap || n > (1 << 30)) return -1;
  p.ntiles = (int)n;
  const int G = grid < p.ntiles ? grid : p.ntiles;     // as tc::launch clamps it
  for (int t = 0; t < p.ntiles; ++t) {
    const TileInfo ti = decode_order(p, t, G);
    out[3 * t] = ti.mt;
    out[3 * t + 1] = ti.nt;
    out[3 * t + 2] = ti.b;
  }
  return p.ntiles;
}
