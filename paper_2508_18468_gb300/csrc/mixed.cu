// Mixed-precision step: placeholder until the tensor-core GEMM lands.
#include "mixed.h"

namespace fm {

bool mixed_supported(int, int, int, std::string* why) {
  *why = "mixed precision path not built";
  return false;
}
size_t mixed_scratch_bytes(int, int, int) { return 0; }
int mixed_init(cudaStream_t, int, int, int, void*, std::string*) { return 1; }
int mixed_step(MixedCtx* c) {
  c->err = "mixed precision path not built";
  return FM_EINVAL;
}
bool mixed_entropy_gram(cudaStream_t, const z64*, int, int, z64*) { return false; }

}  // namespace fm
