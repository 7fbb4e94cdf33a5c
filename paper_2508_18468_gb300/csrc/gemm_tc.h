// Split-fp16 tcgen05 GEMM: host interface.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace fm {
namespace tc {

constexpr int BM = 128;  // tile rows (TMEM lanes)
constexpr int BK = 64;   // K per pipeline stage: one 128-byte swizzle row of fp16

enum Mode {
  MODE_PLAIN = 0,  // out_f[m + n ld_out] = D (fp32)
  MODE_PROP = 1,   // propagation: out_f as PLAIN + per-row sums of D^2 into partial
  MODE_GRAM = 2,   // Gram: D into the real (part 0) / imaginary (part 1) half of complex64 G_b
  MODE_TRMM = 3,   // U R^-1: D into V_b (fp32) and its fp16 planes
  MODE_ADDV = 4,   // out_f[b stride + m + n ld_out] = in_f[same] + D, and its fp16 planes out_h, out_l
  MODE_CPLX = 5    // complex C = alpha D + beta C: the A rows stack the real (row tiles < mt_mod) and
                   // imaginary parts; out_c complex64, ld_out / out_batch_stride in complex elements
};

// Tile orders when Params::tiles is NULL (each a bijection onto the launch's tiles):
enum Order {
  ORDER_RASTER = 0,   // groups of 16 row tiles sweep all column tiles
  ORDER_PAIRS_A = 1,  // triangular A (kb_lo_mt / kb_hi_mt): row blocks mr and mt_mod - 1 - mr, whose
                      //   K ranges add up to a constant, fall to one CTA in consecutive rounds
                      //   (mt_mod even)
  ORDER_PAIRS_B = 2,  // triangular B (kb_hi_nt): the same with column tiles nt and ntiles_n - 1 - nt
                      //   (ntiles_n even)
  ORDER_HERM = 3      // herm_upper: only the tiles mr <= nt (ntiles = batch 2 mt_mod (mt_mod + 1) / 2),
                      //   groups of 16 row tiles sweeping their columns
};

struct Params {
  int mode;
  int order;           // Order (with tiles == NULL)
  int ntiles;
  const int4* tiles;   // (mt, nt, b, part) per tile, device memory; NULL: grouped raster over
  int mtiles, ntiles_n;  //   mtiles x ntiles_n tiles per batch item (batch = ntiles / (mtiles ntiles_n))
  int chunk_kb;        // >0 (BN = 128 only): drain TMEM into fp32 registers every chunk_kb K-blocks
  int64_t out_batch_stride;  // PLAIN: elements between batch items of out_f
  const float* in_f;   // TRMM: if set, out = in + D (D = U (T - 1)); ADDV: the array D is added to
  int kblocks;         // K / BK
  int tri_k;           // limit K-blocks to (nt+1) BN / BK (triangular B)
  // K-block bounds by tile for triangular operands (0: off), with mr = mt % mt_mod:
  int kb_lo_mt;        //   start at mr kb_lo_mt (A upper triangular)
  int kb_hi_mt;        //   end at (mr + 1) kb_hi_mt (A lower triangular)
  int kb_hi_nt;        //   end at (nt + 1) kb_hi_nt (B^T upper triangular)
  int mt_mod;          //   row tiles per block of A rows (the complex embedding stacks Re and Im rows)
  int herm_upper;      // skip the tiles with mr > nt (a Hermitian product's lower tiles)
  int a_rows_per_b;    // A row offset per batch item
  int b_rows_per_b;    // B row offset per batch item
  int k_shift;         // part 1 of the Gram: B read at (k + k_shift) mod kdim, negated past the wrap
  int kdim;            // K in elements
  float* out_f;
  __half* out_h;
  __half* out_l;
  float* out_gf;       // GRAM: complex64 G_b (interleaved re, im)
  double* partial;
  int64_t ld_out;
  int L, Ntraj, C;
  int* status;
  // GRAM: if set, per batch item b the largest |G_kl| over the off-diagonal entries the
  // launch computes, atomically max-ed into estat[2 b + 1] as float bits (G is then a
  // Gram of nearly orthonormal columns, so these are the entries of E = G - 1)
  unsigned* estat;
  // if set and *cond == 0 the launch does nothing (a conditional pass decided on the device)
  const int* cond;
  float* out_c;        // CPLX: complex64 C (interleaved re, im)
  float alpha, beta;   // CPLX
};

bool make_kmajor_map(CUtensorMap* m, const __half* base, uint64_t K, uint64_t rows, uint64_t ld, uint32_t box_rows);
cudaError_t launch(cudaStream_t st, int BN, const CUtensorMap& Ah, const CUtensorMap& Al, const CUtensorMap& Bh,
                   const CUtensorMap& Bl, const Params& p, int grid);
std::vector<int4> tile_list(int mtiles, int ntiles, int batch, int parts, bool upper_only, int BN, int GM);
size_t smem_bytes(int BN);
// shared-memory opt-in of every kernel instantiation (idempotent)
cudaError_t configure_all();
int sm_count();

}  // namespace tc
}  // namespace fm
