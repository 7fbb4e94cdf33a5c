// Entanglement entropy of a caller-held state without any device allocation.
//
// Some callers cannot call cudaMalloc: an application whose own memory pool
// already holds nearly all of the device memory (a fresh cudaMalloc would
// fail), or a latency-sensitive loop that must not pay the device-wide
// synchronisation that freeing memory implies.  For them, the scratch of this
// entry point lives in one fixed array in the library's static device memory,
// which every GPU that loads the library keeps until the process exits.
#include <algorithm>
#include <mutex>

#include "fm.h"
#include "kernels.h"

namespace {

constexpr int kMaxRows = FM_NOALLOC_MAX_SITES;   // largest subsystem
constexpr int kMaxN = FM_NOALLOC_MAX_N;          // largest particle number
constexpr int kMaxM = kMaxN;                     // eigenproblem size min(n, N) <= N

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kRowsOff = 0;
constexpr size_t kMOff = kRowsOff + al((size_t)kMaxRows * kMaxN * 16);
constexpr size_t kVbOff = kMOff + al((size_t)kMaxM * kMaxM * 16);
constexpr size_t kWbOff = kVbOff + al((size_t)kMaxM * 16);
constexpr size_t kPbOff = kWbOff + al((size_t)kMaxM * 16);
constexpr size_t kDOff = kPbOff + al((size_t)fm::hermitian_entropy_pbuf(kMaxM) * 16);
constexpr size_t kEOff = kDOff + al((size_t)kMaxM * 8);
constexpr size_t kLamOff = kEOff + al((size_t)kMaxM * 8);
constexpr size_t kTotal = kLamOff + al((size_t)kMaxM * 8);

// The scratch itself.  In host code this name is only a stand-in, never a
// device address; the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char fm_noalloc_scratch[kTotal];

// The subsystem's sites travel inside the gather kernel's parameters (4 KB, within the
// 32 KB parameter space of current GPUs), so the call makes no host-to-device copy.
struct SiteList {
  int32_t s[kMaxRows];
};

// rows[a + k n] = U[site_a + k L]: the rows of A, n x N column-major.
__global__ void gather_sites_kernel(const z64* __restrict__ U, int L, int N, const SiteList sl, int n,
                                    z64* __restrict__ rows) {
  const int64_t tot = (int64_t)n * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % n);
    const int64_t k = idx / n;
    rows[idx] = U[sl.s[a] + k * L];
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device.
fm_status scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FM_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, fm_noalloc_scratch) != cudaSuccess || !p) return FM_ECUDA;
    g_addr[dev] = p;
  }
  *out = (unsigned char*)g_addr[dev];
  return FM_OK;
}

}  // namespace

extern "C" fm_status fm_entropy_noalloc(const void* d_U, int32_t L, int32_t N, const int32_t* sites, int32_t n,
                                        double* d_S, void* cuda_stream) {
  using namespace fm;
  if (!d_U || !d_S || L < 2 || L > 65536 || N < 1 || N > L || N > kMaxN || n < 0 || n > L || n > kMaxRows ||
      (n > 0 && !sites))
    return FM_EINVAL;
  {
    // distinct, in-range sites, checked on the host with a bitmap on the stack
    uint32_t seen[65536 / 32] = {0};
    for (int i = 0; i < n; ++i) {
      const int j = sites[i];
      if (j < 0 || j >= L) return FM_EINVAL;
      if (seen[j >> 5] & (1u << (j & 31))) return FM_EINVAL;
      seen[j >> 5] |= 1u << (j & 31);
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (n == 0) return cudaMemsetAsync(d_S, 0, sizeof(double), st) == cudaSuccess ? FM_OK : FM_ECUDA;
  unsigned char* base = nullptr;
  fm_status r = scratch_address(&base);
  if (r != FM_OK) return r;
  z64* rows = (z64*)(base + kRowsOff);
  z64* M = (z64*)(base + kMOff);
  z64* vb = (z64*)(base + kVbOff);
  z64* wb = (z64*)(base + kWbOff);
  z64* pb = (z64*)(base + kPbOff);
  double* d = (double*)(base + kDOff);
  double* e = (double*)(base + kEOff);
  double* lam = (double*)(base + kLamOff);
  // Every scratch word read below is written first in the same call, so no
  // clearing is needed between calls.
  SiteList sl;
  for (int i = 0; i < n; ++i) sl.s[i] = sites[i];
  const int64_t tot = (int64_t)n * N;
  const unsigned grid = (unsigned)std::min<int64_t>((tot + 255) / 256, 4 * 152);
  gather_sites_kernel<<<grid, 256, 0, st>>>((const z64*)d_U, L, N, sl, n, rows);
  if (cudaGetLastError() != cudaSuccess) return FM_ECUDA;
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  const int m = n <= N ? n : N;
  cudaError_t ce = (n <= N)
                       ? zgemm<double>(st, n, n, N, OP_N, OP_C, one, rows, n, 0, rows, n, 0, zero, M, n, 0, 1, 0)
                       : zgemm<double>(st, N, N, n, OP_C, OP_N, one, rows, n, 0, rows, n, 0, zero, M, N, 0, 1, 0);
  if (ce != cudaSuccess) return FM_ECUDA;
  if (hermitian_entropy(st, M, m, vb, wb, pb, nullptr, d, e, lam, d_S, nullptr) != cudaSuccess) return FM_ECUDA;
  return FM_OK;
}
