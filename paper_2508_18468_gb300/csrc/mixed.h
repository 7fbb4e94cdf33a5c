// Mixed-precision (split-fp16 tensor-core) step of the fm library.
#pragma once

#include <string>

#include "kernels.h"
#include "timer.h"

namespace fm {

// Device pointers and step parameters of one state (filled at init; V / V2
// swap as the step double-buffers the float state).
struct MixedCtx {
  cudaStream_t st;
  int Lx, Ly, L, N, B;
  int protocol, reorth_interval;
  int tile_config;         // fm_params.tile_config (validated)
  double dt, J;
  uint64_t seed;
  int64_t global_step;
  float *V, *V2;           // state (2L x N float per trajectory) and its double buffer
  __half *Vh, *Vl;         // split-fp16 planes of V (x = h + l 2^-11)
  __half *Ah, *Al;         // planes of the real 2L x 2L propagator embedding (row-major)
  __half *Th, *Tl;         // planes of the real 2N x 2N embedding of R^-1, K-major (per trajectory)
  z64 *G, *R, *T, *Dinv, *X;
  double* gamma; uint64_t* traj; int64_t* step; int* status;
  double *part, *nocc, *w;
  void *xbuf, *vbuf;
  fm_event* log; int64_t* log_count; int log_capacity;
  const int4* force; int force_n;   // forced projective outcomes (sorted), n = 0: none
  void* extra;             // mixed_scratch_bytes() of device scratch
  PhaseTimer* timer;       // phase events (may be off)
  void* pmw;               // scratch of the grid-wide projective update
  int prop_banded;         // propagation as stencils (fm_set_propagation)
  const z64 *band_tx, *band_ty;   // taps along x and y (device)
  const int *band_ox, *band_oy;   // their site offsets
  int ntap_x, ntap_y;
  float* rk4buf;           // Runge-Kutta stage buffer (FM_HOMODYNE_RK4)
  int64_t launches;        // out: kernels launched
  std::string err;         // out: message on failure
};

struct MixedHost;          // tensor maps and tile lists of one state

bool mixed_supported(int Lx, int Ly, int batch, int tile_config, std::string* why);
size_t mixed_scratch_bytes(int Lx, int Ly, int batch, int protocol);
MixedHost* mixed_create(MixedCtx* c, std::string* why);   // uploads tile lists, encodes tensor maps
void mixed_free(MixedHost* h);
int mixed_step(MixedHost* h, MixedCtx* c);               // returns an fm_status value
int mixed_reorth(MixedHost* h, MixedCtx* c);             // fp16 planes of V, then both CholeskyQR passes
// the second CholeskyQR pass (and its guard's extra pass) on the current state, the
// product written back into V (the buffers stay put): completes a step period early
int mixed_settle(MixedHost* h, MixedCtx* c);
// second-pass guard: counts[0] passes checked, counts[1] extra passes run (since init);
// maxima[0..3] the largest |diag E|, |offdiag E| measured by the second passes and by the
// extra passes since the previous call (which then restart from zero).  Synchronises st.
int mixed_guard_stats(MixedHost* h, cudaStream_t st, int64_t* counts, double* maxima);

}  // namespace fm
