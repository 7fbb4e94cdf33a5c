// C ABI of the fm library: state, workspace plan, step orchestration.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <complex>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fm.h"
#include "kernels.h"
#include "mixed.h"
#include "timer.h"

using namespace fm;

namespace {

const int kCholNB = CHOL_NB;   // Cholesky / triangular-inverse block
const int kMaxChunks = 128;    // occupation partial sums
const int kAsyncSlots = 64;    // outstanding asynchronous entropies
// C_A buffers of the asynchronous entropies: as many as fit in 4 GiB, 4 to 64 (many
// small trajectories then keep their tickets in flight together)
const int kEaRingMax = 64;
// library threads of the asynchronous entropies: as many as fit their scratch in 1 GiB, 1
// to 4 (small eigen-solves are latency-bound: several run side by side)
const int kEaWorkersMax = 4;
const int kEaIssuedCap = 256;   // > outstanding tickets (64 results, 64 C_A buffers)
int ea_ring_size(int64_t N) {
  const int64_t per = 16 * N * N;
  return (int)std::max<int64_t>(4, std::min<int64_t>(kEaRingMax, (int64_t(4) << 30) / std::max<int64_t>(per, 1)));
}
const int kPoisSlots = 128;    // continuous-time projective: propagation slots per upload
// entropy sketch (FM_EE_SKETCH): first rank, power iterations, convergence bound on the
// (r/8)-th smallest Ritz value sigma^2, smallest subsystem (and complement) it is used for
const int kSketchR0 = 128;
const int kSketchQ = 1;
const double kSketchTol = 1e-9;
const int kSketchMinSites = 4 * kSketchR0;
// FM_EE_AUTO takes the sketch from here on: measured at l = 512 the full method takes
// 21 ms and the sketch 30 ms (its float64 bases are latency-bound at that size), at
// l = 8192 the full method 5.5 s and the sketch 0.06 s
const int kSketchAutoSites = 1024;
int sketch_rmax(int64_t N) { return N >= kSketchMinSites ? (int)std::min<int64_t>(1024, (N / 2) / 32 * 32) : 0; }

// continuous-time projective scratch: taps (slot, trajectory, x then y), event
// sites and draws (trajectory, slot), event counts, then the tap offsets
int64_t pois_al(int64_t x) { return (x + 255) & ~(int64_t)255; }
int64_t pois_bytes(int64_t B) {
  return pois_al(kPoisSlots * B * 2 * kBandMaxTaps * 16) + pois_al(kPoisSlots * B * 4) + pois_al(kPoisSlots * B * 8) +
         pois_al(B * 4) + pois_al(2 * kBandMaxTaps * 4);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Plan {
  size_t total = 0;
  // offsets
  size_t gamma, traj, step, status, occ, log_count, log, force, part, nocc, w, xbuf, vbuf;
  size_t U, U2, P, G, R, T, Dinv, X;                  // FP64 path (G, R, T, Dinv, X also mixed)
  size_t V, V2, Vh, Vl, Ah, Al, Th, Tl, aux;           // mixed path
  size_t ee_vb, ee_wb, ee_pb, ee_d, ee_e, ee_lam, ee_S, ee_sites, ee_max;
  size_t chk_cols, chk_G;                               // orthonormality check (<= 64 columns)
  size_t ea_M, ea_vb, ea_wb, ea_pb, ea_d, ea_e, ea_lam, ea_S;   // asynchronous entropy (ea_vb .. ea_lam per worker)
  int ea_workers = 1;
  size_t pmw;                                           // grid-wide projective update
  size_t xg;                                            // exact-product Gram of C_A (mixed)
  size_t gfull;                                         // exact Gram of all of U (mixed)
  size_t obs;                                           // displacement bins and partial sums
  size_t band;                                          // stencil taps and offsets (x, y)
  size_t rk4;                                           // Runge-Kutta stage buffer
  size_t pois;                                          // continuous-time projective: taps, offsets
  size_t sk_snap, sk_sync, sk_async, sk_res;            // entropy sketch (mixed)
  size_t mixed_extra;                                   // scratch owned by the mixed path
  size_t take(size_t bytes) { size_t o = total; total += align256(bytes); return o; }
};

bool valid_params(const fm_params* p, std::string* why) {
  if (!p) { *why = "params is NULL"; return false; }
  if (p->Lx < 2 || p->Ly < 1) { *why = "need Lx >= 2, Ly >= 1"; return false; }
  const int64_t L = (int64_t)p->Lx * p->Ly;
  if (L % 2) { *why = "L = Lx*Ly must be even (half filling)"; return false; }
  if (p->Ly > 1 && (p->Lx % 2)) { *why = "torus needs even Lx for the checkerboard start"; return false; }
  if (L > 65536) { *why = "L > 65536 not supported"; return false; }
  if (p->batch < 1 || p->batch > 65535) { *why = "batch must be in [1, 65535]"; return false; }
  if (p->protocol != FM_PROJECTIVE && p->protocol != FM_HOMODYNE && p->protocol != FM_HOMODYNE_RK4 &&
      p->protocol != FM_PROJECTIVE_POISSON) {
    *why = "bad protocol";
    return false;
  }
  if (p->precision != FM_FP64 && p->precision != FM_MIXED) { *why = "bad precision"; return false; }
  if (p->reorth_interval < 1) { *why = "reorth_interval must be >= 1"; return false; }
  if (p->event_capacity < 0) { *why = "event_capacity must be >= 0"; return false; }
  if (!(p->dt > 0.0) || !isfinite(p->J) || !(p->gamma >= 0.0) || !isfinite(p->gamma)) {
    *why = "need dt > 0, finite J, gamma >= 0";
    return false;
  }
  if (p->precision == FM_MIXED) {
    std::string w2;
    if (!mixed_supported(p->Lx, p->Ly, p->batch, p->tile_config, &w2)) { *why = w2; return false; }
  }
  return true;
}

// library threads of the asynchronous entropies for these parameters (kEaWorkersMax at most)
int ea_workers(const fm_params& p) {
  const int64_t L = (int64_t)p.Lx * p.Ly, N = L / 2;
  int64_t per = 2 * N * 16 + hermitian_entropy_pbuf((int)N) * 16 + 3 * N * 8;
  const int rmax = p.precision == FM_MIXED ? sketch_rmax(N) : 0;
  if (rmax) per += (int64_t)sketch_scratch_bytes((int)L, (int)N, rmax);
  return (int)std::max<int64_t>(1, std::min<int64_t>(kEaWorkersMax, (int64_t(1) << 30) / std::max<int64_t>(per, 1)));
}

Plan make_plan(const fm_params& p) {
  Plan pl;
  const int64_t L = (int64_t)p.Lx * p.Ly, N = L / 2, B = p.batch;
  const int64_t nblk = (N + kCholNB - 1) / kCholNB;
  pl.gamma = pl.take(B * 8);
  pl.traj = pl.take(B * 8);
  pl.step = pl.take(B * 8);
  pl.status = pl.take(16);
  pl.occ = pl.take(N * 4);
  pl.log_count = pl.take(16);
  pl.log = pl.take((size_t)p.event_capacity * sizeof(fm_event));
  pl.force = pl.take((size_t)p.event_capacity * 16);
  pl.part = pl.take(B * kMaxChunks * L * 8);
  pl.nocc = pl.take(B * L * 8);
  pl.w = pl.take(B * L * 8);
  pl.xbuf = pl.take(B * N * 16);
  pl.vbuf = pl.take(B * L * 16);
  // float64 CholeskyQR factors of every trajectory (FP64 path); the mixed path keeps its
  // factors in its own scratch and uses G only as one N x N matrix (entropy, covariance)
  const int64_t nf = p.precision == FM_FP64 ? B : 0;
  pl.G = pl.take(std::max<int64_t>(nf, 1) * N * N * 16);
  pl.R = pl.take(nf * N * N * 16);
  pl.T = pl.take(nf * N * N * 16);
  pl.Dinv = pl.take(nf * nblk * kCholNB * kCholNB * 16);
  pl.X = pl.take(nf * N * kCholNB * 16);
  pl.ee_vb = pl.take(N * 16);
  pl.ee_wb = pl.take(N * 16);
  pl.ee_pb = pl.take(std::max<int64_t>(hermitian_entropy_pbuf((int)N), 1 + 32 * N) * 16);
  pl.ee_d = pl.take(N * 8);
  pl.ee_e = pl.take(N * 8);
  pl.ee_lam = pl.take(N * 8);
  pl.ee_S = pl.take(8);
  pl.ee_max = pl.take(8);
  pl.ee_sites = pl.take(L * 4);
  pl.chk_cols = pl.take(L * std::min<int64_t>(N, 64) * 16);
  pl.chk_G = pl.take(std::min<int64_t>(N, 64) * N * 16);
  pl.ea_M = pl.take(ea_ring_size(N) * N * N * 16);
  pl.ea_workers = ea_workers(p);
  pl.ea_vb = pl.take(pl.ea_workers * N * 16);
  pl.ea_wb = pl.take(pl.ea_workers * N * 16);
  pl.ea_pb = pl.take(pl.ea_workers * hermitian_entropy_pbuf((int)N) * 16);
  pl.ea_d = pl.take(pl.ea_workers * N * 8);
  pl.ea_e = pl.take(pl.ea_workers * N * 8);
  pl.ea_lam = pl.take(pl.ea_workers * N * 8);
  pl.ea_S = pl.take(kAsyncSlots * 8);
  pl.pmw = pl.take(pm_wide_scratch_bytes((int)L, (int)B));
  pl.obs = pl.take((L + abs2_partials() + 8) * 8);
  pl.band = pl.take(2 * kBandMaxTaps * (16 + 4));
  pl.rk4 = pl.take(p.protocol == FM_HOMODYNE_RK4 ? B * L * N * (p.precision == FM_FP64 ? 16 : 8) : 0);
  pl.pois = pl.take(p.protocol == FM_PROJECTIVE_POISSON ? pois_bytes(B) : 0);
  if (p.precision == FM_FP64) {
    pl.U = pl.take(B * L * N * 16);
    pl.U2 = pl.take(B * L * N * 16);
    pl.P = pl.take(L * L * 16);
    pl.aux = pl.U2;
  } else {
    pl.V = pl.take(B * 2 * L * N * 4);
    pl.V2 = pl.take(B * 2 * L * N * 4);
    pl.Vh = pl.take(B * 2 * L * N * 2);
    pl.Vl = pl.take(B * 2 * L * N * 2);
    pl.Ah = pl.take(4 * L * L * 2);
    pl.Al = pl.take(4 * L * L * 2);
    pl.Th = pl.take(B * 4 * N * N * 2);
    pl.Tl = pl.take(B * 4 * N * N * 2);
    pl.aux = pl.take(L * N * 16);
    pl.mixed_extra = pl.take(mixed_scratch_bytes(p.Lx, p.Ly, p.batch, p.protocol));
    pl.xg = pl.take(std::max(exact_gram_scratch_bytes((int)L, (int)N), projector_scratch_bytes((int)N)));
    pl.gfull = pl.take(N * N * 16);
    const int rmax = sketch_rmax(N);
    if (rmax) {
      pl.sk_snap = pl.take(L * N * 8);
      pl.sk_sync = pl.take(sketch_scratch_bytes((int)L, (int)N, rmax));
      pl.sk_async = pl.take(pl.ea_workers * align256(sketch_scratch_bytes((int)L, (int)N, rmax)));
    }
    pl.sk_res = pl.take(64);
  }
  return pl;
}

}  // namespace

struct fm_state {
  fm_params prm;
  int Lx, Ly, L, N, B;
  cudaStream_t st;
  char* ws;
  size_t ws_bytes;
  Plan pl;
  // common
  double* gamma_d; uint64_t* traj_d; int64_t* step_d; int* status_d; int* occ_d;
  unsigned long long* log_count_d; fm_event* log_d;
  int4* force_d; int force_n;   // forced projective outcomes (fm_force_outcomes), sorted
  double *part_d, *nocc_d, *w_d;
  void *xbuf_d, *vbuf_d;
  z64 *G, *R, *T, *Dinv, *X;
  // fp64
  z64 *U, *U2, *P;
  // mixed
  float *V, *V2;
  __half *Vh, *Vl, *Ah, *Al, *Th, *Tl;
  z64* aux;
  void* mixed_extra;
  void* xg;                  // exact-product Gram scratch (mixed precision)
  z64* gfull;                // exact Gram of all of U, for the projector correction
  MixedCtx mc;
  MixedHost* mh;
  PhaseTimer timer;
  // CUDA graph of one step period
  bool graphs_on;
  cudaStream_t cap_st;
  cudaGraphExec_t graph_exec;
  int graph_period;
  int64_t graph_launch_count;
  // EE
  z64 *ee_vb, *ee_wb, *ee_pb;
  double *ee_d, *ee_e, *ee_lam, *ee_S, *ee_max;
  int* ee_sites;
  z64 *chk_cols, *chk_G;
  // Asynchronous entropy.  The caller's thread gathers the rows of A and
  // forms C_A on the caller's stream (into one of ea_ring buffers); a library
  // thread issues the eigen-solver launches (about 5 per row of C_A) on a
  // low-priority stream.  Steps then run on a high-priority stream bridged to
  // the caller's by events, so the FP64 eigen-solve fills what the steps'
  // kernels leave of each SM and the caller's thread never waits on the
  // launch queue.
  int dev;
  z64* ea_M;                  // ea_ring x N x N
  int ea_ring;
  // one library thread per worker, each with its own low-priority stream and scratch
  struct EaWorker {
    std::thread th;
    cudaStream_t st = nullptr;
    z64 *vb, *wb, *pb;
    double *d, *e, *lam, *chk;
    SketchScratch sk;
  };
  int ea_nw;
  EaWorker ea_w[kEaWorkersMax];
  double* ea_S;
  cudaStream_t ea_st, hp_st;  // ea_st: worker 0's stream
  cudaEvent_t hp_in, hp_out;
  cudaEvent_t ea_M_ready[kEaRingMax], ea_M_free[kEaRingMax];
  cudaEvent_t ea_done[kAsyncSlots];
  double* ea_host;            // pinned, kAsyncSlots doubles
  void* pmw;                  // grid-wide projective update scratch
  double* obs;                // displacement bins, partial sums, one result
  // structured propagation (fm_set_propagation): stencil taps per direction
  int prop_mode;
  z64 *band_tx, *band_ty;
  int *band_ox, *band_oy;
  int ntap_x, ntap_y;
  void* rk4buf;               // Runge-Kutta stage buffer (FM_HOMODYNE_RK4)
  // continuous-time projective protocol: next event index and time per trajectory,
  // device taps (slot, trajectory, x then y) and the common offsets of each direction
  std::vector<int64_t> pois_e;
  std::vector<double> pois_t;
  z64* pois_taps;
  int* pois_list;              // B x kPoisSlots sites of a chunk of slots
  double* pois_u;              // their Born draws
  int* pois_cnt;               // events of each trajectory in the chunk
  int* pois_off;               // x offsets, then y offsets (kBandMaxTaps each)
  int pois_wx, pois_wy;        // half-widths; -1: every offset of that direction
  // entropy method (fm_set_entropy_method) and the sketch's buffers: a snapshot of U
  // with A's rows first for the synchronous path (asynchronous tickets keep theirs in
  // their C_A ring buffer), one scratch set per path, and device results
  int ee_method;
  int sk_rmax;
  c32* sk_snap;
  SketchScratch sk_sync;
  double* sk_res;             // [0] S, [1] check (synchronous); [2 + w] check (library thread w)
  int sk_last_rank;
  double sk_last_chk;
  int sk_last_fallback;
  // aux, gfull and xg are shared by the caller's thread (the full method) and the
  // library thread (the full method after a sketch that did not converge): a user
  // holds ee_buf_mu while it enqueues and orders its stream after ee_buf_ev
  std::mutex ee_buf_mu;
  cudaEvent_t ee_buf_ev;
  int64_t ea_next;            // next ticket
  struct EaJob { int64_t t; int slot, ring, m, sketch_nA; };   // sketch_nA > 0: the ring holds a snapshot
  std::vector<char> ea_issued_flag;   // tickets done, by ticket % kEaIssuedCap
  std::mutex ea_mu;
  std::condition_variable ea_cv;
  std::deque<EaJob> ea_q;
  int64_t ea_issued;          // every ticket below it has all its launches enqueued
  bool ea_stop;
  bool ea_failed;
  std::string ea_errmsg;
  std::atomic<int64_t> ea_launches;
  // host
  std::vector<double> gamma_h;
  std::vector<uint64_t> traj_h;
  std::vector<int64_t> step_h;
  int64_t global_steps;
  int64_t settled_step;       // global step at which the pending second pass last ran early (-1: never)
  int64_t config_gen;         // bumped whenever captured step graphs of this state go stale
  int sticky;
  std::string err;
  int64_t launches;
};

namespace {

// Record an error.  Device / numeric failures are sticky; argument errors are not.
fm_status fail(fm_state* s, fm_status code, const std::string& msg) {
  if (s && !s->sticky) {
    s->err = msg;
    if (code == FM_ECUDA || code == FM_ENUMERIC || code == FM_ETIMEOUT) s->sticky = code;
  }
  return code;
}

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(s, FM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

#define CKL(call, n)                                                                             \
  do {                                                                                           \
    CK(call);                                                                                    \
    s->launches += (n);                                                                          \
  } while (0)

// Read and clear the device status word; map to a sticky error.
fm_status sync_and_check(fm_state* s) {
  CK(cudaStreamSynchronize(s->st));
  int st = 0;
  CK(cudaMemcpy(&st, s->status_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    int zero = 0;
    CK(cudaMemcpy(s->status_d, &zero, sizeof(int), cudaMemcpyHostToDevice));
    if (st & FM_DEVERR_TIMEOUT) return fail(s, FM_ETIMEOUT, "a bounded device wait gave up");
    if (st & FM_DEVERR_PIVOT) return fail(s, FM_ENUMERIC, "non-positive Cholesky pivot (U lost rank)");
    if (st & FM_DEVERR_NONFINITE) return fail(s, FM_ENUMERIC, "non-finite values in U");
    if (st & FM_DEVERR_REORTH)
      return fail(s, FM_ENUMERIC, "re-orthonormalisation did not converge (U^dag U - 1 still above the "
                                  "first-order pass's reach after the extra pass)");
    return fail(s, FM_ENUMERIC, "device error flag " + std::to_string(st));
  }
  return FM_OK;
}

// p[r] = (1/L) sum_m exp(2 pi i m r / L) exp(-2 i J dt cos(2 pi m / L)), the
// angle index m*r reduced mod L exactly (plane-wave form of exp(-i H~ dt)).
std::vector<z64> ring_row(int L, double J, double dt) {
  std::vector<z64> out(L);
  if (L == 1) { out[0].re = 1.0; out[0].im = 0.0; return out; }
  std::vector<double> c(L), sn(L);
  for (int q = 0; q < L; ++q) {
    const double a = 2.0 * M_PI * (double)q / (double)L;
    c[q] = cos(a);
    sn[q] = sin(a);
  }
  std::vector<std::complex<double>> ph(L);
  for (int m = 0; m < L; ++m) ph[m] = std::exp(std::complex<double>(0.0, -2.0 * J * dt * c[m]));
  for (int r = 0; r < L; ++r) {
    std::complex<double> acc(0.0, 0.0);
    int64_t q = 0;
    for (int m = 0; m < L; ++m) {
      acc += std::complex<double>(c[q], sn[q]) * ph[m];
      q += r;
      if (q >= L) q -= L;
    }
    acc /= (double)L;
    out[r].re = acc.real();
    out[r].im = acc.imag();
  }
  return out;
}

std::vector<int> occupied(int Lx, int Ly) {
  std::vector<int> occ;
  for (int y = 0; y < Ly; ++y)
    for (int x = 0; x < Lx; ++x) {
      const bool on = (Ly == 1) ? (x % 2 == 0) : ((x + y) % 2 == 0);
      if (on) occ.push_back(x + Lx * y);
    }
  return occ;
}

// Stencil of one direction of the circulant propagator row p (length n): the
// offsets up to the half-width beyond which every tap is below 1e-15 (the
// plane-wave sums that give p carry rounding noise of ~1e-17, so a smaller
// cut would keep noise); every offset when that width reaches half the period.
void band_taps(const std::vector<z64>& p, std::vector<z64>* taps, std::vector<int>* off) {
  const int n = (int)p.size();
  auto mag = [&](int r) { const z64 z = p[((r % n) + n) % n]; return sqrt(z.re * z.re + z.im * z.im); };
  int w = 0;
  for (int r = 1; r <= n / 2; ++r)
    if (mag(r) > 1e-15 || mag(-r) > 1e-15) w = r;
  taps->clear();
  off->clear();
  if (2 * w + 1 >= n) {
    for (int r = 0; r < n; ++r) { taps->push_back(p[r]); off->push_back(r); }
  } else {
    for (int r = -w; r <= w; ++r) { taps->push_back(p[((r % n) + n) % n]); off->push_back(r); }
  }
}

// ------------------------------------------------------------------ continuous-time projective protocol
// Philox4x32-10 on the host (Salmon et al., SC'11), for the event draws the host
// needs to schedule the propagation between events.
std::array<uint32_t, 4> philox_host(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return {c0, c1, c2, c3};
}
double u53_host(uint32_t wa, uint32_t wb) {
  return ((double)(wa >> 5) * 67108864.0 + (double)(wb >> 6)) * (1.0 / 9007199254740992.0);
}
struct PoisDraw { double u_wait; int site; double u; };
PoisDraw poisson_draw(uint64_t seed, uint64_t traj, int64_t e, int L) {
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  const uint32_t c0 = (uint32_t)((uint64_t)e & 0xFFFFFFFFu), c1 = (uint32_t)((uint64_t)e >> 32);
  const uint32_t c2 = (uint32_t)(traj & 0xFFFFFFFFu), hi = (uint32_t)(traj >> 32) << 8;
  const auto w = philox_host(c0, c1, c2, 3u | hi, k0, k1);
  const auto v = philox_host(c0, c1, c2, 4u | hi, k0, k1);
  PoisDraw d;
  d.u_wait = u53_host(w[0], w[1]);
  d.site = std::min((int)(u53_host(w[2], w[3]) * L), L - 1);
  d.u = u53_host(v[0], v[1]);
  return d;
}
// taps of exp(-i H~ tau) along one direction of length n: at the offsets -w .. w
// from the Jacobi-Anger series, p_r = (-i)^|r| J_|r|(2 J tau) (the aliased terms
// J_{n - |r|} are below 1e-17 wherever this form is used), or (w < 0) at every
// offset 0 .. n-1 from the plane-wave sum
void poisson_taps(int n, int w, double J, double tau, z64* out) {
  if (w < 0) {
    std::vector<z64> row = ring_row(n, J, tau);
    for (int r = 0; r < n; ++r) out[r] = row[r];
    return;
  }
  static const double re4[4] = {1.0, 0.0, -1.0, 0.0}, im4[4] = {0.0, -1.0, 0.0, 1.0};  // (-i)^r
  const double z = 2.0 * std::fabs(J) * tau;
  for (int t = 0; t <= 2 * w; ++t) {
    const int r = std::abs(t - w);
    double jr = std::cyl_bessel_j((double)r, z);
    if (J < 0.0 && (r & 1)) jr = -jr;            // J_r(-z) = (-1)^r J_r(z)
    out[t].re = re4[r % 4] * jr;
    out[t].im = im4[r % 4] * jr;
  }
}

// half-width of that stencil for every tau <= dt along a direction of length n
// (J_r(2 |J| tau) grows with tau for r > 2 |J| tau): -1 when 2w + 1 reaches n
int poisson_width(int n, double J, double dt) {
  const double z = 2.0 * std::fabs(J) * dt;
  int w = 0;
  for (; w < 4 * kBandMaxTaps; ++w) {
    bool small = w + 1 > z;
    for (int r = w + 1; small && r <= w + 8; ++r) small = std::fabs(std::cyl_bessel_j((double)r, z)) < 1e-17;
    if (small) break;
  }
  return 2 * w + 1 >= n ? -1 : w;
}

double poisson_wait(const fm_state* s, int b, int64_t e) {
  const double rate = s->gamma_h[b] * (double)s->N;
  if (!(rate > 0.0)) return INFINITY;
  return -std::log1p(-poisson_draw(s->prm.seed, s->traj_h[b], e, s->L).u_wait) / rate;
}

// index and time of trajectory b's next event at its step count: the events up to
// step_h[b] dt replayed (the running sum of the waiting times)
void poisson_sync(fm_state* s, int b) {
  int64_t e = 0;
  double t = poisson_wait(s, b, 0);
  if (s->step_h[b] > 0) {
    const double t0 = (double)s->step_h[b] * s->prm.dt;
    while (t <= t0) {
      ++e;
      t = t + poisson_wait(s, b, e);
    }
  }
  s->pois_e[b] = e;
  s->pois_t[b] = t;
}

fm_status poisson_setup(fm_state* s) {
  const double J = s->prm.J, dt = s->prm.dt;
  s->pois_wx = poisson_width(s->Lx, J, dt);
  s->pois_wy = s->Ly > 1 ? poisson_width(s->Ly, J, dt) : -1;
  const int ntx = s->pois_wx < 0 ? s->Lx : 2 * s->pois_wx + 1;
  const int nty = s->pois_wy < 0 ? s->Ly : 2 * s->pois_wy + 1;
  if (ntx > kBandMaxTaps || nty > kBandMaxTaps)
    return fail(s, FM_EINVAL, "continuous-time protocol: J dt too large for the stencil propagation");
  std::vector<int> off(2 * kBandMaxTaps, 0);
  for (int t = 0; t < ntx; ++t) off[t] = s->pois_wx < 0 ? t : t - s->pois_wx;
  for (int t = 0; t < nty; ++t) off[kBandMaxTaps + t] = s->pois_wy < 0 ? t : t - s->pois_wy;
  CK(cudaMemcpyAsync(s->pois_off, off.data(), 4 * off.size(), cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  s->pois_e.assign(s->B, 0);
  s->pois_t.assign(s->B, 0.0);
  for (int b = 0; b < s->B; ++b) poisson_sync(s, b);
  return FM_OK;
}

fm_status check_state(fm_state* s) {
  if (!s) return FM_EINVAL;
  if (s->sticky) return FM_ESTATE;
  return FM_OK;
}

// A mixed-precision state whose step period is not complete (reorth_interval k > 1 and
// the last step not a multiple of k) has had only the first CholeskyQR pass since its
// last second pass: U^dag U - 1 is then ~1e-6..1e-5 instead of < 1e-7.  Observables
// that read U first run that pending second pass now (in place: the buffers a captured
// step graph uses stay put); span(U), the state itself, does not change.  The steps that
// follow continue the usual k-step schedule.
fm_status settle(fm_state* s) {
  if (!s->mh || s->prm.reorth_interval <= 1 || s->global_steps % s->prm.reorth_interval == 0 ||
      s->settled_step == s->global_steps)
    return FM_OK;
  MixedCtx& c = s->mc;
  c.st = s->st;
  c.V = s->V; c.V2 = s->V2;
  c.launches = 0;
  fm_status r = (fm_status)mixed_settle(s->mh, &c);
  s->launches += c.launches;
  if (r) return fail(s, r, c.err);
  s->settled_step = s->global_steps;
  return FM_OK;
}

// ------------------------------------------------------------------ FP64 CholeskyQR pass
// G = U^dag U ; G = R^dag R ; T = R^-1 ; U <- U T
fm_status cholqr_f64(fm_state* s) {
  const int L = s->L, N = s->N, B = s->B;
  const int64_t sNN = (int64_t)N * N, sLN = (int64_t)L * N;
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  s->timer.begin(FM_PH_GRAM);
  CKL(zgemm<double>(s->st, N, N, L, OP_C, OP_N, one, s->U, L, sLN, s->U, L, sLN, zero, s->G, N, sNN, B,
                    GEMM_UPPER_ONLY), 1);
  s->timer.end(FM_PH_GRAM);
  s->timer.begin(FM_PH_CHOLESKY);
  CK(cholesky_inverse<double>(s->st, s->G, s->R, s->T, s->Dinv, s->X, N, N, sNN, N, B, s->status_d, &s->launches));
  s->timer.end(FM_PH_CHOLESKY);
  s->timer.begin(FM_PH_TRMM);
  CKL(zgemm<double>(s->st, L, N, N, OP_N, OP_N, one, s->U, L, sLN, s->T, N, sNN, zero, s->U2, L, sLN, B,
                    GEMM_TRI_B_UPPER), 1);
  s->timer.end(FM_PH_TRMM);
  std::swap(s->U, s->U2);
  s->aux = s->U2;
  return FM_OK;
}

fm_status step_f64(fm_state* s) {
  const int L = s->L, N = s->N, B = s->B;
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  if (s->prm.protocol == FM_HOMODYNE_RK4) {
    // App. A's integrator: <n> of U(t), the weights' logarithms, four Horner stages
    const int nch = occupation_chunks(L, N, B);
    s->timer.begin(FM_PH_MEASURE);
    CKL(rownorm_partials_z(s->st, s->U, L, N, B, s->part_d, nch), 1);
    CKL(reduce_occupations(s->st, s->part_d, nch, L, B, s->nocc_d, s->w_d, s->gamma_d, s->prm.dt, s->traj_d,
                           s->step_d, s->prm.seed), 1);
    s->timer.end(FM_PH_MEASURE);
    s->timer.begin(FM_PH_PROPAGATE);
    const double h = s->prm.dt * s->prm.J;
    void* R4 = s->rk4buf;
    CKL(rk4_stage(s->st, 0, s->U, s->U, R4, L, N, B, s->Lx, s->Ly, s->w_d, h, 0.25), 1);
    CKL(rk4_stage(s->st, 0, s->U, R4, s->U2, L, N, B, s->Lx, s->Ly, s->w_d, h, 1.0 / 3.0), 1);
    CKL(rk4_stage(s->st, 0, s->U, s->U2, R4, L, N, B, s->Lx, s->Ly, s->w_d, h, 0.5), 1);
    CKL(rk4_stage(s->st, 0, s->U, R4, s->U2, L, N, B, s->Lx, s->Ly, s->w_d, h, 1.0), 1);
    s->timer.end(FM_PH_PROPAGATE);
    std::swap(s->U, s->U2);
    s->aux = s->U2;
    fm_status r = cholqr_f64(s);
    if (r) return r;
    if ((s->global_steps + 1) % s->prm.reorth_interval == 0 && (r = cholqr_f64(s))) return r;
    CKL(bump_steps(s->st, s->step_d, B), 1);
    return FM_OK;
  }
  // 1. propagation, all trajectories in one product P [U_0 | U_1 | ...], or as stencils
  s->timer.begin(FM_PH_PROPAGATE);
  if (s->prop_mode == FM_PROP_BANDED) {
    CKL(band_propagate(s->st, 0, s->U, s->U2, L, N, B, s->Lx, s->Ly, 0, s->band_tx, s->band_ox, s->ntap_x, nullptr,
                       band_chunks(s->Lx, s->Ly, N, B, 0, 0)), 1);
    if (s->Ly > 1) {
      CKL(band_propagate(s->st, 0, s->U2, s->U, L, N, B, s->Lx, s->Ly, 1, s->band_ty, s->band_oy, s->ntap_y,
                         nullptr, band_chunks(s->Lx, s->Ly, N, B, 1, 0)), 1);
    } else {
      std::swap(s->U, s->U2);
    }
  } else {
    CKL(zgemm<double>(s->st, L, N * B, L, OP_N, OP_N, one, s->P, L, 0, s->U, L, 0, zero, s->U2, L, 0, 1, 0), 1);
    std::swap(s->U, s->U2);
  }
  s->timer.end(FM_PH_PROPAGATE);
  s->aux = s->U2;
  const int64_t gstep = s->global_steps;
  const int k = s->prm.reorth_interval;
  if (s->prm.protocol == FM_HOMODYNE) {
    const int nch = occupation_chunks(L, N, B);
    s->timer.begin(FM_PH_MEASURE);
    CKL(rownorm_partials_z(s->st, s->U, L, N, B, s->part_d, nch), 1);
    CKL(reduce_occupations(s->st, s->part_d, nch, L, B, s->nocc_d, s->w_d, s->gamma_d, s->prm.dt, s->traj_d,
                           s->step_d, s->prm.seed), 1);
    CKL(scale_rows_z(s->st, s->U, L, N, B, s->w_d), 1);
    s->timer.end(FM_PH_MEASURE);
    fm_status r = cholqr_f64(s);
    if (r) return r;
    if ((gstep + 1) % k == 0) {
      r = cholqr_f64(s);
      if (r) return r;
    }
  } else {
    pm_args a;
    a.U = s->U; a.L = L; a.N = N; a.batch = B; a.layout = 0;
    a.gamma = s->gamma_d; a.dt = s->prm.dt; a.traj = s->traj_d; a.step = s->step_d; a.seed = s->prm.seed;
    a.xbuf = s->xbuf_d; a.vbuf = s->vbuf_d;
    a.log = s->log_d; a.log_count = (int64_t*)s->log_count_d; a.log_capacity = s->prm.event_capacity;
    a.dev_status = s->status_d;
    a.force = s->force_d; a.force_n = s->force_n;
    s->timer.begin(FM_PH_MEASURE);
    if (pm_use_wide(L, N, B)) CK(pm_measure_wide(s->st, a, s->pmw, &s->launches));
    else CKL(pm_measure(s->st, a), 1);
    s->timer.end(FM_PH_MEASURE);
    if ((gstep + 1) % k == 0) {
      fm_status r = cholqr_f64(s);
      if (r) return r;
      r = cholqr_f64(s);
      if (r) return r;
    }
  }
  CKL(bump_steps(s->st, s->step_d, B), 1);
  return FM_OK;
}

// One step of the continuous-time projective protocol (App. A), all trajectories.
// The host draws each trajectory's events in (t, t + dt] (the waiting times need
// no state) and lays the step out in slots: slot q propagates every trajectory
// by its q-th interval (the time to its q-th event, then the rest of the step,
// then zero) as two stencils with per-trajectory taps, and applies the q-th
// event of every trajectory that has one (row and Born weight, v = U x^dag,
// rank-1 update).  Taps and events go up in chunks of kPoisSlots slots.
fm_status step_poisson(fm_state* s) {
  const int L = s->L, N = s->N, B = s->B;
  const double dt = s->prm.dt, J = s->prm.J;
  const bool fp64 = s->prm.precision == FM_FP64;
  const int ntx = s->pois_wx < 0 ? s->Lx : 2 * s->pois_wx + 1;
  const int nty = s->pois_wy < 0 ? s->Ly : 2 * s->pois_wy + 1;
  const int tstride = ntx + (s->Ly > 1 ? nty : 0);
  // the schedule: intervals (events + 1) and events per trajectory
  std::vector<std::vector<double>> tau(B);
  std::vector<std::vector<int>> site(B);
  std::vector<std::vector<double>> uo(B);
  int kmax = 0;
  for (int b = 0; b < B; ++b) {
    const double t1 = (double)(s->step_h[b] + 1) * dt;
    double t = (double)s->step_h[b] * dt;
    while (s->pois_t[b] <= t1) {
      const PoisDraw d = poisson_draw(s->prm.seed, s->traj_h[b], s->pois_e[b], L);
      tau[b].push_back(s->pois_t[b] - t);
      site[b].push_back(d.site);
      uo[b].push_back(d.u);
      t = s->pois_t[b];
      s->pois_e[b] += 1;
      s->pois_t[b] = s->pois_t[b] + poisson_wait(s, b, s->pois_e[b]);
    }
    tau[b].push_back(t1 - t);
    kmax = std::max(kmax, (int)site[b].size());
  }
  pm_args a;
  a.L = L; a.N = N; a.batch = B; a.layout = fp64 ? 0 : 1;
  a.gamma = s->gamma_d; a.dt = dt; a.traj = s->traj_d; a.step = s->step_d; a.seed = s->prm.seed;
  a.xbuf = s->xbuf_d; a.vbuf = s->vbuf_d;
  a.log = s->log_d; a.log_count = (int64_t*)s->log_count_d; a.log_capacity = s->prm.event_capacity;
  a.dev_status = s->status_d;
  a.force = nullptr; a.force_n = 0;
  const int nchx = band_chunks(s->Lx, s->Ly, N, B, 0, a.layout), nchy = band_chunks(s->Lx, s->Ly, N, B, 1, a.layout);
  std::vector<z64> taps;
  std::vector<int> list, cnt(B);
  std::vector<double> ul;
  const int nslot = kmax + 1;
  for (int q0 = 0; q0 < nslot; q0 += kPoisSlots) {
    const int S = std::min(kPoisSlots, nslot - q0);
    taps.assign((size_t)S * B * tstride, z64{0.0, 0.0});
    list.assign((size_t)B * S, 0);
    ul.assign((size_t)B * S, 0.0);
    for (int b = 0; b < B; ++b) {
      const int nev = (int)site[b].size();
      cnt[b] = std::max(0, std::min(S, nev - q0));
      for (int j = 0; j < S; ++j) {
        const int q = q0 + j;
        const double tq = q < (int)tau[b].size() ? tau[b][q] : 0.0;
        z64* tp = taps.data() + ((size_t)j * B + b) * tstride;
        poisson_taps(s->Lx, s->pois_wx, J, tq, tp);
        if (s->Ly > 1) poisson_taps(s->Ly, s->pois_wy, J, tq, tp + ntx);
        if (q < nev) {
          list[(size_t)b * S + j] = site[b][q];
          ul[(size_t)b * S + j] = uo[b][q];
        }
      }
    }
    // pageable sources: each copy returns once its bytes are staged, so the vectors
    // may be refilled (next chunk) or freed (end of the step) at once
    s->timer.begin(FM_PH_MEASURE);
    CK(cudaMemcpyAsync(s->pois_taps, taps.data(), 16 * taps.size(), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->pois_list, list.data(), 4 * list.size(), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->pois_u, ul.data(), 8 * ul.size(), cudaMemcpyHostToDevice, s->st));
    CK(cudaMemcpyAsync(s->pois_cnt, cnt.data(), 4 * B, cudaMemcpyHostToDevice, s->st));
    s->timer.end(FM_PH_MEASURE);
    for (int j = 0; j < S; ++j) {
      void* cur = fp64 ? (void*)s->U : (void*)s->V;
      void* oth = fp64 ? (void*)s->U2 : (void*)s->V2;
      const z64* tp = s->pois_taps + (size_t)j * B * tstride;
      s->timer.begin(FM_PH_PROPAGATE);
      CKL(band_propagate(s->st, a.layout, cur, oth, L, N, B, s->Lx, s->Ly, 0, tp, s->pois_off, ntx, nullptr, nchx,
                         tstride), 1);
      if (s->Ly > 1) {
        CKL(band_propagate(s->st, a.layout, oth, cur, L, N, B, s->Lx, s->Ly, 1, tp + ntx, s->pois_off + kBandMaxTaps,
                           nty, nullptr, nchy, tstride), 1);
      } else if (fp64) {
        std::swap(s->U, s->U2);
      } else {
        std::swap(s->V, s->V2);
      }
      s->timer.end(FM_PH_PROPAGATE);
      if (q0 + j < kmax) {
        a.U = fp64 ? (void*)s->U : (void*)s->V;
        s->timer.begin(FM_PH_MEASURE);
        CKL(pm_wide_event(s->st, a, j, s->pois_list, s->pois_u, S, s->pois_cnt, s->pmw), 3);
        s->timer.end(FM_PH_MEASURE);
      }
    }
  }
  if (fp64) s->aux = s->U2;
  if ((s->global_steps + 1) % s->prm.reorth_interval == 0) {
    if (fp64) {
      fm_status r = cholqr_f64(s);
      if (r) return r;
      if ((r = cholqr_f64(s))) return r;
    } else {
      MixedCtx& c = s->mc;
      c.st = s->st;
      c.V = s->V; c.V2 = s->V2;
      c.launches = 0;
      const int r = mixed_reorth(s->mh, &c);
      s->V = c.V; s->V2 = c.V2;
      s->launches += c.launches;
      if (r) return fail(s, (fm_status)r, c.err);
    }
  }
  CKL(bump_steps(s->st, s->step_d, B), 1);
  return FM_OK;
}

fm_status validate_sites(fm_state* s, const int32_t* sites, int32_t n) {
  if (n < 0 || n > s->L || (n > 0 && !sites)) return fail(s, FM_EINVAL, "bad site list");
  std::vector<char> seen(s->L, 0);
  for (int i = 0; i < n; ++i) {
    if (sites[i] < 0 || sites[i] >= s->L) return fail(s, FM_EINVAL, "site index out of range");
    if (seen[sites[i]]) return fail(s, FM_EINVAL, "repeated site in subsystem");
    seen[sites[i]] = 1;
  }
  return FM_OK;
}

// C_A (or U_A^dag U_A when n > N, the same nonzero spectrum) of trajectory b for
// the n sites in d_sites (device) into M on stream st; only the lower triangle
// when the eigen-solver reads only that.  FP64 state: the FP64 product of the
// gathered rows.  Mixed precision (float state), large blocks: exact digit
// products on the tensor cores, then the first-order correction from U U^dag to
// the projector onto span(U) (the float U is orthonormal only to ~1e-7), which
// needs the exact Gram of all of U first.
fm_status form_correlation(fm_state* s, cudaStream_t st, int b, const int* d_sites, int n, z64* M) {
  const int L = s->L, N = s->N;
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  const int m = std::min(n, N);
  const int fl = hermitian_entropy_lower_only(m) ? GEMM_LOWER_ONLY : 0;
  if (s->prm.precision == FM_MIXED && hermitian_entropy_lower_only(m)) {
    const float* Vb = s->V + (int64_t)b * 2 * L * N;
    CKL(v_to_z(st, Vb, L, N, s->aux), 1);
    CK(exact_gram(st, s->aux, L, N, s->gfull, s->xg, s->status_d, &s->launches));
    CKL(gather_rows_v(st, Vb, L, N, d_sites, n, s->aux), 1);
    CK(exact_gram(st, s->aux, n, N, M, s->xg, s->status_d, &s->launches));
    CK(projector_correct(st, s->gfull, s->aux, n, N, M, s->xg, &s->launches));
    return FM_OK;
  }
  if (s->prm.precision == FM_FP64) {
    CKL(gather_rows_z(st, s->U + (int64_t)b * L * N, L, N, d_sites, n, s->aux), 1);
  } else {
    CKL(gather_rows_v(st, s->V + (int64_t)b * 2 * L * N, L, N, d_sites, n, s->aux), 1);
  }
  if (n <= N) {
    CKL(zgemm<double>(st, n, n, N, OP_N, OP_C, one, s->aux, n, 0, s->aux, n, 0, zero, M, n, 0, 1, fl), 1);
  } else {
    CKL(zgemm<double>(st, N, N, n, OP_C, OP_N, one, s->aux, n, 0, s->aux, n, 0, zero, M, N, 0, 1, fl), 1);
  }
  return FM_OK;
}

// ---- shared buffers of the full method (aux, gfull, xg): see fm_state::ee_buf_mu
void buf_acquire(fm_state* s, cudaStream_t st) {
  s->ee_buf_mu.lock();
  if (s->ee_buf_ev) cudaStreamWaitEvent(st, s->ee_buf_ev, 0);
}
void buf_release(fm_state* s, cudaStream_t st) {
  if (s->ee_buf_ev) cudaEventRecord(s->ee_buf_ev, st);
  s->ee_buf_mu.unlock();
}

struct BufGuard {
  fm_state* s;
  cudaStream_t st;
  BufGuard(fm_state* s_, cudaStream_t st_) : s(s_), st(st_) { buf_acquire(s, st); }
  ~BufGuard() { buf_release(s, st); }
};

bool sketch_applicable(const fm_state* s, int n) {
  const int side = std::min(n, s->L - n);
  if (s->sk_rmax == 0) return false;
  if (s->ee_method == FM_EE_SKETCH) return side >= kSketchMinSites;
  if (s->ee_method == FM_EE_AUTO) return side >= kSketchAutoSites;
  return false;
}

// sites of A (as given), then the rest in ascending order, into the device list
fm_status upload_permutation(fm_state* s, const int32_t* sites, int32_t n) {
  std::vector<int> perm(sites, sites + n);
  std::vector<char> in(s->L, 0);
  for (int i = 0; i < n; ++i) in[sites[i]] = 1;
  for (int i = 0; i < s->L; ++i)
    if (!in[i]) perm.push_back(i);
  CK(cudaMemcpyAsync(s->ee_sites, perm.data(), sizeof(int) * s->L, cudaMemcpyHostToDevice, s->st));
  // the pageable source is staged before the call returns
  return FM_OK;
}

// The adaptive sketch on `st` over a snapshot (A's rows first, ld L): ranks kSketchR0,
// 2 kSketchR0, ... while below both side sizes and sk_rmax.  Returns 1 when converged (S
// at S_dev), 0 when not, -1 on a CUDA error (message in *err).
int run_sketch(fm_state* s, cudaStream_t st, const c32* snap, int nA, const SketchScratch& w, double* S_dev,
               double* chk_dev, int64_t* launches, int* rank, double* chk, std::string* err) {
  const int nB = s->L - nA;
  const uint64_t seed = s->prm.seed ^ 0x5eedc0de5eedc0deull;
  *rank = 0;
  *chk = 0.0;
  for (int r = kSketchR0; r <= s->sk_rmax && r < std::min(nA, nB); r *= 2) {
    cudaError_t e = sketch_entropy(st, snap, s->L, nA, nB, s->N, r, kSketchQ, seed, w, S_dev, chk_dev, launches);
    double c = 0.0;
    int stat = 0;
    if (!e) e = cudaMemcpyAsync(&c, chk_dev, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaMemcpyAsync(&stat, w.status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (!e) e = cudaStreamSynchronize(st);
    if (e) {
      *err = std::string("entropy sketch: ") + cudaGetErrorString(e);
      return -1;
    }
    *rank = r;
    *chk = c;
    if (stat == 0 && std::isfinite(c) && c <= kSketchTol) return 1;
  }
  return 0;
}

// S_A of trajectory b; enqueues and synchronises.  Uses its own scratch, so
// asynchronous entropies still in flight are not disturbed.
fm_status entropy_impl(fm_state* s, int b, const int32_t* sites, int32_t n, double* S_out) {
  if (n == 0) { *S_out = 0.0; return FM_OK; }
  fm_status r;
  s->timer.begin(FM_PH_ENTROPY);
  if (sketch_applicable(s, n)) {
    if ((r = upload_permutation(s, sites, n))) return r;
    CKL(gather_rows_c32(s->st, s->V + (int64_t)b * 2 * s->L * s->N, s->L, s->N, s->ee_sites, s->L, s->sk_snap), 1);
    std::string err;
    const int c = run_sketch(s, s->st, s->sk_snap, n, s->sk_sync, s->sk_res, s->sk_res + 1, &s->launches,
                             &s->sk_last_rank, &s->sk_last_chk, &err);
    if (c < 0) return fail(s, FM_ECUDA, err);
    s->sk_last_fallback = c == 0;
    if (c == 1) {
      s->timer.end(FM_PH_ENTROPY);
      CK(cudaMemcpyAsync(S_out, s->sk_res, sizeof(double), cudaMemcpyDeviceToHost, s->st));
      return sync_and_check(s);
    }
    // not converged: the full method below (the list still starts with A's sites)
  } else {
    CK(cudaMemcpyAsync(s->ee_sites, sites, sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
    if (s->ee_method != FM_EE_FULL) {
      s->sk_last_rank = 0;
      s->sk_last_chk = 0.0;
      s->sk_last_fallback = 1;
    }
  }
  z64* M = s->G;  // scratch between steps
  buf_acquire(s, s->st);
  r = form_correlation(s, s->st, b, s->ee_sites, n, M);
  buf_release(s, s->st);
  if (r) return r;
  int nl = 0;
  CK(hermitian_entropy(s->st, M, std::min(n, s->N), s->ee_vb, s->ee_wb, s->ee_pb, nullptr, s->ee_d, s->ee_e,
                       s->ee_lam, s->ee_S, &nl));
  s->launches += nl;
  s->timer.end(FM_PH_ENTROPY);
  CK(cudaMemcpyAsync(S_out, s->ee_S, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

// one eager step of the whole batch on s->st
fm_status step_once(fm_state* s) {
  fm_status r;
  if (s->prm.protocol == FM_PROJECTIVE_POISSON) r = step_poisson(s);
  else if (s->prm.precision == FM_FP64) r = step_f64(s);
  else {
    MixedCtx& c = s->mc;
    c.st = s->st;
    c.global_step = s->global_steps;
    c.V = s->V; c.V2 = s->V2;
    c.launches = 0;
    r = (fm_status)mixed_step(s->mh, &c);
    s->V = c.V; s->V2 = c.V2;
    s->launches += c.launches;
    if (r) r = fail(s, r, c.err);
  }
  if (r) return r;
  s->global_steps += 1;
  for (int b = 0; b < s->B; ++b) s->step_h[b] += 1;
  return FM_OK;
}

// Whether the steps of s can be captured into a graph: host-scheduled steps (event
// counts read back: the grid-wide projective path and the mixed-precision projective
// block; events drawn on the host: the continuous-time protocol) cannot.
bool graph_capable(const fm_state* s) {
  if (s->prm.protocol == FM_PROJECTIVE_POISSON) return false;
  if (s->prm.protocol == FM_PROJECTIVE && (s->mh || pm_use_wide(s->L, s->N, s->B))) return false;
  return true;
}

// Issue P steps of s on stream cs (which is being captured); nothing executes, so the
// host bookkeeping is restored afterwards.  *per: the launches of the P steps.
fm_status issue_period(fm_state* s, cudaStream_t cs, int P, int64_t* per) {
  cudaStream_t user = s->st;
  const int64_t g0 = s->global_steps;
  const int64_t l0 = s->launches;
  std::vector<int64_t> steps0 = s->step_h;
  z64* U0 = s->U;
  float* V0 = s->V;
  const bool timing = s->timer.on;
  s->timer.on = false;
  s->st = cs;
  s->timer.st = cs;
  fm_status r = FM_OK;
  for (int i = 0; i < P && r == FM_OK; ++i) r = step_once(s);
  s->st = user;
  s->timer.st = user;
  s->timer.on = timing;
  if (s->prm.precision != FM_FP64) s->mc.st = user;
  *per = s->launches - l0;
  s->global_steps = g0;
  s->step_h = steps0;
  s->launches = l0;
  if (r == FM_OK && (s->U != U0 || s->V != V0)) r = fail(s, FM_ECUDA, "graph period does not return the state buffers");
  return r;
}

// Capture one period of steps into s->graph_exec (state pointers return to
// their starting buffers after a period, so the graph can be replayed).
fm_status capture_period(fm_state* s) {
  if (!s->cap_st) CK(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
  CK(cudaStreamSynchronize(s->st));
  fm_status r = FM_OK;
  cudaGraph_t graph = nullptr;
  int64_t per_period = 0;
  if (cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    r = fail(s, FM_ECUDA, "cudaStreamBeginCapture");
  } else {
    r = issue_period(s, s->cap_st, s->graph_period, &per_period);
    cudaError_t e = cudaStreamEndCapture(s->cap_st, &graph);
    if (r == FM_OK && e != cudaSuccess) r = fail(s, FM_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
  }
  if (r == FM_OK) {
    if (cudaGraphInstantiate(&s->graph_exec, graph, 0) != cudaSuccess) r = fail(s, FM_ECUDA, "cudaGraphInstantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  s->graph_launch_count = per_period;
  return r;
}

// nsteps steps on s->st: eager up to the next period boundary, then whole
// periods as CUDA-graph replays when graphs are on, eager for the rest
fm_status step_many(fm_state* s, int32_t nsteps) {
  fm_status r;
  int i = 0;
  if (s->graphs_on && graph_capable(s)) {
    const int P = s->graph_period;
    while (i < nsteps && (s->global_steps % P) != 0) {
      if ((r = step_once(s))) return r;
      ++i;
    }
    while (nsteps - i >= P) {
      if (!s->graph_exec && (r = capture_period(s))) return r;
      CK(cudaGraphLaunch(s->graph_exec, s->st));
      s->launches += s->graph_launch_count;
      s->global_steps += P;
      for (int b = 0; b < s->B; ++b) s->step_h[b] += P;
      i += P;
    }
  }
  for (; i < nsteps; ++i)
    if ((r = step_once(s))) return r;
  return FM_OK;
}

// Re-target the state to another tile configuration and reorth interval and
// put every trajectory back in the Neel state at step 0 (the autotuner's loop).
fm_status retune(fm_state* s, int tile_config, int reorth) {
  CK(cudaStreamSynchronize(s->st));
  if (s->graph_exec) {
    cudaGraphExecDestroy(s->graph_exec);
    s->graph_exec = nullptr;
  }
  s->prm.tile_config = tile_config;
  s->prm.reorth_interval = reorth;
  s->graph_period = 2 * reorth;
  const int L = s->L, N = s->N, B = s->B;
  if (s->prm.precision == FM_FP64) {
    CKL(neel_init_z(s->st, s->U, L, N, B, s->occ_d), 1);
  } else {
    mixed_free(s->mh);
    s->mh = nullptr;
    s->mc.tile_config = tile_config;
    s->mc.reorth_interval = reorth;
    s->mc.st = s->st;
    std::string why;
    s->mh = mixed_create(&s->mc, &why);
    if (!s->mh) return fail(s, FM_ECUDA, "mixed re-init: " + why);
    CKL(neel_init_v(s->st, s->V, s->Vh, s->Vl, L, N, B, s->occ_d), 1);
  }
  s->global_steps = 0;
  s->settled_step = -1;
  s->config_gen += 1;
  for (int b = 0; b < B; ++b) s->step_h[b] = 0;
  if (s->prm.protocol == FM_PROJECTIVE_POISSON)
    for (int b = 0; b < B; ++b) poisson_sync(s, b);
  CK(cudaMemsetAsync(s->step_d, 0, 8 * (size_t)B, s->st));
  CK(cudaStreamSynchronize(s->st));
  return FM_OK;
}

// ------------------------------------------------------------------ asynchronous entropy
// The library threads (ea_nw of them, each with its own low-priority stream and
// scratch): for each job, wait for its C_A (or snapshot), run the eigen-solver or the
// sketch on the thread's stream, copy S to the pinned slot and record the slot's event.
// Launch errors are kept for fm_entropy_wait (the state's error fields belong to the
// caller).
// The full method from an asynchronous ticket's snapshot (U, A's nA rows first, ld L,
// complex64) on the library thread: the exact Gram of all rows (the projector
// correction's U^dag U), then C_A of the smaller of A and its complement (the same
// entropy for a pure state), written over the snapshot.  *m: order of that C_A.
cudaError_t sketch_fallback(fm_state* s, cudaStream_t st, z64* slot, int nA, int* m, int64_t* launches) {
  const int L = s->L, N = s->N;
  const int nS = std::min(nA, L - nA), off = nA <= L - nA ? 0 : nA;
  const c32* snap = (const c32*)slot;
  buf_acquire(s, st);
  cudaError_t e = exact_gram_c32(st, snap, L, L, N, s->gfull, s->xg, s->status_d, launches);
  if (!e) e = rows_c32_to_z64(st, snap + off, L, nS, N, s->aux);
  if (!e) ++*launches;
  if (!e) e = exact_gram(st, s->aux, nS, N, slot, s->xg, s->status_d, launches);
  if (!e) e = projector_correct(st, s->gfull, s->aux, nS, N, slot, s->xg, launches);
  buf_release(s, st);
  *m = nS;
  return e;
}

void ea_worker(fm_state* s, int wk) {
  cudaSetDevice(s->dev);
  fm_state::EaWorker& ew = s->ea_w[wk];
  const cudaStream_t st = ew.st;
  for (;;) {
    fm_state::EaJob j;
    {
      std::unique_lock<std::mutex> lk(s->ea_mu);
      s->ea_cv.wait(lk, [s] { return s->ea_stop || !s->ea_q.empty(); });
      if (s->ea_q.empty()) return;          // stop requested and nothing left
      j = s->ea_q.front();
      s->ea_q.pop_front();
    }
    cudaError_t e = cudaStreamWaitEvent(st, s->ea_M_ready[j.ring], 0);
    const char* what = "cudaStreamWaitEvent";
    z64* M = s->ea_M + (int64_t)j.ring * s->N * s->N;
    int m = j.m;
    bool done = false;
    if (e == cudaSuccess && j.m > 0 && j.sketch_nA > 0) {
      int rank = 0;
      double chk = 0.0;
      int64_t nl = 0;
      std::string err;
      const int c = run_sketch(s, st, (const c32*)M, j.sketch_nA, ew.sk, s->ea_S + j.slot, ew.chk, &nl, &rank, &chk,
                               &err);
      s->ea_launches += nl;
      if (c < 0) {
        e = cudaErrorLaunchFailure;
        what = "entropy sketch";
      } else if (c == 1) {
        done = true;
      } else {
        // not converged: C_A of the smaller side from the snapshot, then the full method
        nl = 0;
        e = sketch_fallback(s, st, M, j.sketch_nA, &m, &nl);
        s->ea_launches += nl;
        what = "entropy fallback";
      }
    }
    if (e == cudaSuccess && !done) {
      if (m == 0) {
        e = cudaMemsetAsync(s->ea_S + j.slot, 0, sizeof(double), st);
        what = "cudaMemsetAsync";
      } else {
        int nl = 0;
        e = hermitian_entropy(st, M, m, ew.vb, ew.wb, ew.pb, nullptr, ew.d, ew.e, ew.lam, s->ea_S + j.slot, &nl);
        s->ea_launches += nl;
        what = "eigen-solver launch";
      }
    }
    if (e == cudaSuccess) {
      e = cudaMemcpyAsync(s->ea_host + j.slot, s->ea_S + j.slot, sizeof(double), cudaMemcpyDeviceToHost, st);
      what = "cudaMemcpyAsync";
    }
    if (e == cudaSuccess) e = cudaEventRecord(s->ea_M_free[j.ring], st);
    if (e == cudaSuccess) e = cudaEventRecord(s->ea_done[j.slot], st);
    std::lock_guard<std::mutex> lk(s->ea_mu);
    if (e != cudaSuccess && !s->ea_failed) {
      s->ea_failed = true;
      s->ea_errmsg = std::string("asynchronous entropy: ") + what + ": " + cudaGetErrorString(e);
    }
    // tickets finish out of order across the threads: advance the issued prefix
    s->ea_issued_flag[j.t % kEaIssuedCap] = 1;
    while (s->ea_issued_flag[s->ea_issued % kEaIssuedCap]) {
      s->ea_issued_flag[s->ea_issued % kEaIssuedCap] = 0;
      ++s->ea_issued;
    }
    s->ea_cv.notify_all();
  }
}

fm_status ea_setup(fm_state* s) {
  if (s->ea_st) return FM_OK;
  int least = 0, greatest = 0;
  CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  for (int k = 0; k < s->ea_nw; ++k)
    CK(cudaStreamCreateWithPriority(&s->ea_w[k].st, cudaStreamNonBlocking, least));
  s->ea_st = s->ea_w[0].st;
  CK(cudaStreamCreateWithPriority(&s->hp_st, cudaStreamNonBlocking, greatest));
  CK(cudaEventCreateWithFlags(&s->ee_buf_ev, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->hp_in, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&s->hp_out, cudaEventDisableTiming));
  for (int i = 0; i < s->ea_ring; ++i) {
    CK(cudaEventCreateWithFlags(&s->ea_M_ready[i], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&s->ea_M_free[i], cudaEventDisableTiming));
  }
  for (int i = 0; i < kAsyncSlots; ++i) CK(cudaEventCreateWithFlags(&s->ea_done[i], cudaEventDisableTiming));
  CK(cudaHostAlloc((void**)&s->ea_host, kAsyncSlots * sizeof(double), cudaHostAllocDefault));
  s->ea_stop = false;
  for (int k = 0; k < s->ea_nw; ++k) s->ea_w[k].th = std::thread(ea_worker, s, k);
  return FM_OK;
}

// Block until the library thread has enqueued everything of tickets < t.
void ea_wait_issued(fm_state* s, int64_t t) {
  std::unique_lock<std::mutex> lk(s->ea_mu);
  s->ea_cv.wait(lk, [s, t] { return s->ea_issued >= t; });
}

fm_status ea_check(fm_state* s) {
  std::lock_guard<std::mutex> lk(s->ea_mu);
  if (s->ea_failed) return fail(s, FM_ECUDA, s->ea_errmsg);
  return FM_OK;
}

fm_status entropy_async_impl(fm_state* s, int b, const int32_t* sites, int32_t n, int64_t* ticket) {
  fm_status r = ea_setup(s);
  if (r) return r;
  if ((r = ea_check(s))) return r;
  const int64_t t = s->ea_next;
  const int slot = (int)(t % kAsyncSlots);
  const int ring = (int)(t % s->ea_ring);
  const int N = s->N;
  const int m = std::min(n, N);
  if (t >= kAsyncSlots) {                                   // slot reuse: the oldest result must be back
    ea_wait_issued(s, t - kAsyncSlots + 1);
    CK(cudaEventSynchronize(s->ea_done[slot]));
  }
  z64* M = s->ea_M + (int64_t)ring * N * N;
  int sketch_nA = 0;
  if (m > 0) {
    // C_A buffer reuse: the eigen-solve of ticket t - ea_ring must be queued before
    // the caller's stream may wait for it to release the buffer
    if (t >= s->ea_ring) {
      ea_wait_issued(s, t - s->ea_ring + 1);
      CK(cudaStreamWaitEvent(s->st, s->ea_M_free[ring], 0));
    }
    if (sketch_applicable(s, n)) {
      // U with A's rows first into the C_A buffer (16 N^2 bytes either way), in order
      // with the steps; the library thread runs the sketch on it
      if ((r = upload_permutation(s, sites, n))) return r;
      CKL(gather_rows_c32(s->st, s->V + (int64_t)b * 2 * s->L * N, s->L, N, s->ee_sites, s->L, (c32*)M), 1);
      sketch_nA = n;
    } else {
      // rows of A and C_A, in order with the steps on the caller's stream
      CK(cudaMemcpyAsync(s->ee_sites, sites, sizeof(int) * n, cudaMemcpyHostToDevice, s->st));
      buf_acquire(s, s->st);
      r = form_correlation(s, s->st, b, s->ee_sites, n, M);
      buf_release(s, s->st);
      if (r) return r;
    }
  }
  CK(cudaEventRecord(s->ea_M_ready[ring], s->st));
  {
    std::lock_guard<std::mutex> lk(s->ea_mu);
    s->ea_q.push_back(fm_state::EaJob{t, slot, ring, m, sketch_nA});
  }
  s->ea_cv.notify_all();
  s->ea_next = t + 1;
  *ticket = t;
  return FM_OK;
}

}  // namespace

// =================================================================== public API
extern "C" {

const char* fm_version(void) { return "fm 0.1 (sm_103a)"; }

size_t fm_workspace_bytes(const fm_params* p) {
  std::string why;
  if (!valid_params(p, &why)) return 0;
  return make_plan(*p).total;
}

fm_status fm_init_state(const fm_params* p, void* d_workspace, size_t ws_bytes, void* cuda_stream, fm_state** out) {
  if (!out) return FM_EINVAL;
  *out = nullptr;
  std::string why;
  if (!valid_params(p, &why)) return FM_EINVAL;
  Plan pl = make_plan(*p);
  if (!d_workspace || ((uintptr_t)d_workspace & 255)) return FM_EINVAL;
  if (ws_bytes < pl.total) return FM_ENOMEM;
  fm_state* s = new fm_state();
  s->prm = *p;
  s->Lx = p->Lx; s->Ly = p->Ly; s->L = p->Lx * p->Ly; s->N = s->L / 2; s->B = p->batch;
  s->st = (cudaStream_t)cuda_stream;
  s->ws = (char*)d_workspace; s->ws_bytes = ws_bytes; s->pl = pl;
  s->global_steps = 0; s->sticky = 0; s->launches = 0;
  s->graphs_on = false; s->cap_st = nullptr; s->graph_exec = nullptr; s->graph_period = 0;
  s->settled_step = -1;
  s->config_gen = 0;
  char* w = s->ws;
  s->gamma_d = (double*)(w + pl.gamma); s->traj_d = (uint64_t*)(w + pl.traj); s->step_d = (int64_t*)(w + pl.step);
  s->status_d = (int*)(w + pl.status); s->occ_d = (int*)(w + pl.occ);
  s->log_count_d = (unsigned long long*)(w + pl.log_count); s->log_d = (fm_event*)(w + pl.log);
  s->force_d = (int4*)(w + pl.force); s->force_n = 0;
  s->part_d = (double*)(w + pl.part); s->nocc_d = (double*)(w + pl.nocc); s->w_d = (double*)(w + pl.w);
  s->xbuf_d = w + pl.xbuf; s->vbuf_d = w + pl.vbuf;
  s->G = (z64*)(w + pl.G); s->R = (z64*)(w + pl.R); s->T = (z64*)(w + pl.T);
  s->Dinv = (z64*)(w + pl.Dinv); s->X = (z64*)(w + pl.X);
  if (p->precision != FM_FP64) s->R = s->T = s->Dinv = s->X = nullptr;   // not allocated
  s->ee_vb = (z64*)(w + pl.ee_vb); s->ee_wb = (z64*)(w + pl.ee_wb); s->ee_pb = (z64*)(w + pl.ee_pb);
  s->ee_d = (double*)(w + pl.ee_d); s->ee_e = (double*)(w + pl.ee_e); s->ee_lam = (double*)(w + pl.ee_lam);
  s->ee_S = (double*)(w + pl.ee_S); s->ee_max = (double*)(w + pl.ee_max); s->ee_sites = (int*)(w + pl.ee_sites);
  s->chk_cols = (z64*)(w + pl.chk_cols); s->chk_G = (z64*)(w + pl.chk_G);
  s->ea_M = (z64*)(w + pl.ea_M);
  s->ea_nw = pl.ea_workers;
  for (int k = 0; k < s->ea_nw; ++k) {
    fm_state::EaWorker& ew = s->ea_w[k];
    const int64_t Nn = p->Lx * (int64_t)p->Ly / 2;
    ew.vb = (z64*)(w + pl.ea_vb) + k * Nn;
    ew.wb = (z64*)(w + pl.ea_wb) + k * Nn;
    ew.pb = (z64*)(w + pl.ea_pb) + k * hermitian_entropy_pbuf((int)Nn);
    ew.d = (double*)(w + pl.ea_d) + k * Nn;
    ew.e = (double*)(w + pl.ea_e) + k * Nn;
    ew.lam = (double*)(w + pl.ea_lam) + k * Nn;
  }
  s->ea_issued_flag.assign(kEaIssuedCap, 0);
  s->ea_S = (double*)(w + pl.ea_S);
  s->ea_st = s->hp_st = nullptr; s->hp_in = s->hp_out = nullptr; s->ea_host = nullptr; s->ea_next = 0;
  s->ea_ring = ea_ring_size(s->N);
  for (int i = 0; i < kEaRingMax; ++i) s->ea_M_ready[i] = s->ea_M_free[i] = nullptr;
  s->ea_issued = 0; s->ea_stop = false; s->ea_failed = false; s->ea_launches = 0;
  if (cudaGetDevice(&s->dev) != cudaSuccess) { delete s; return FM_ECUDA; }
  s->pmw = w + pl.pmw;
  s->obs = (double*)(w + pl.obs);
  s->prop_mode = FM_PROP_DENSE;
  s->band_tx = (z64*)(w + pl.band);
  s->band_ty = s->band_tx + kBandMaxTaps;
  s->band_ox = (int*)(s->band_ty + kBandMaxTaps);
  s->band_oy = s->band_ox + kBandMaxTaps;
  s->ntap_x = s->ntap_y = 0;
  s->rk4buf = w + pl.rk4;
  s->ee_method = FM_EE_FULL;
  s->sk_rmax = p->precision == FM_MIXED ? sketch_rmax(p->Lx * (int64_t)p->Ly / 2) : 0;
  s->sk_snap = nullptr;
  if (s->sk_rmax) {
    const int Lh = p->Lx * p->Ly, Nh = Lh / 2;
    s->sk_snap = (c32*)(w + pl.sk_snap);
    s->sk_sync = sketch_layout(w + pl.sk_sync, Lh, Nh, s->sk_rmax);
    const size_t skb = align256(sketch_scratch_bytes(Lh, Nh, s->sk_rmax));
    for (int k = 0; k < s->ea_nw; ++k) s->ea_w[k].sk = sketch_layout(w + pl.sk_async + k * skb, Lh, Nh, s->sk_rmax);
  }
  s->sk_res = (double*)(w + pl.sk_res);
  for (int k = 0; k < s->ea_nw; ++k) s->ea_w[k].chk = s->sk_res + 2 + k;
  s->sk_last_rank = 0; s->sk_last_chk = 0.0; s->sk_last_fallback = 0;
  s->ee_buf_ev = nullptr;
  {
    char* q = w + pl.pois;
    const int64_t B = p->batch;
    s->pois_taps = (z64*)q;
    q += pois_al(kPoisSlots * B * 2 * kBandMaxTaps * 16);
    s->pois_list = (int*)q;
    q += pois_al(kPoisSlots * B * 4);
    s->pois_u = (double*)q;
    q += pois_al(kPoisSlots * B * 8);
    s->pois_cnt = (int*)q;
    q += pois_al(B * 4);
    s->pois_off = (int*)q;
  }
  for (int i = 0; i < kAsyncSlots; ++i) s->ea_done[i] = nullptr;
  s->U = s->U2 = s->P = nullptr; s->V = s->V2 = nullptr;
  s->Vh = s->Vl = s->Ah = s->Al = s->Th = s->Tl = nullptr;
  s->mixed_extra = nullptr;
  s->xg = nullptr;
  s->gfull = nullptr;
  s->mh = nullptr;
  if (p->precision == FM_FP64) {
    s->U = (z64*)(w + pl.U); s->U2 = (z64*)(w + pl.U2); s->P = (z64*)(w + pl.P); s->aux = s->U2;
  } else {
    s->V = (float*)(w + pl.V); s->V2 = (float*)(w + pl.V2);
    s->Vh = (__half*)(w + pl.Vh); s->Vl = (__half*)(w + pl.Vl);
    s->Ah = (__half*)(w + pl.Ah); s->Al = (__half*)(w + pl.Al);
    s->Th = (__half*)(w + pl.Th); s->Tl = (__half*)(w + pl.Tl);
    s->aux = (z64*)(w + pl.aux); s->mixed_extra = w + pl.mixed_extra; s->xg = w + pl.xg;
    s->gfull = (z64*)(w + pl.gfull);
  }
  s->timer.st = s->st;
  s->gamma_h.assign(s->B, p->gamma);
  s->traj_h.resize(s->B);
  for (int b = 0; b < s->B; ++b) s->traj_h[b] = p->traj_id + (uint64_t)b;
  s->step_h.assign(s->B, 0);

  fm_status r = FM_OK;
  do {
    // zero the whole workspace once: triangular factors rely on zero lower parts
    if (cudaMemsetAsync(s->ws, 0, pl.total, s->st) != cudaSuccess) { r = fail(s, FM_ECUDA, "memset"); break; }
    if (cudaMemcpyAsync(s->gamma_d, s->gamma_h.data(), 8 * s->B, cudaMemcpyHostToDevice, s->st) ||
        cudaMemcpyAsync(s->traj_d, s->traj_h.data(), 8 * s->B, cudaMemcpyHostToDevice, s->st)) {
      r = fail(s, FM_ECUDA, "upload");
      break;
    }
    std::vector<int> occ = occupied(s->Lx, s->Ly);
    if ((int)occ.size() != s->N) { r = fail(s, FM_EINVAL, "checkerboard does not half fill"); break; }
    if (cudaMemcpyAsync(s->occ_d, occ.data(), 4 * s->N, cudaMemcpyHostToDevice, s->st)) {
      r = fail(s, FM_ECUDA, "upload occ");
      break;
    }
    std::vector<z64> px = ring_row(s->Lx, p->J, p->dt), py = ring_row(s->Ly, p->J, p->dt);
    {
      std::vector<z64> tx, ty;
      std::vector<int> ox, oy;
      band_taps(px, &tx, &ox);
      band_taps(py, &ty, &oy);
      if ((int)tx.size() > kBandMaxTaps || (int)ty.size() > kBandMaxTaps) {
        s->ntap_x = s->ntap_y = 0;   // too wide a stencil: dense propagation only
      } else {
        s->ntap_x = (int)tx.size();
        s->ntap_y = (int)ty.size();
        if (cudaMemcpyAsync(s->band_tx, tx.data(), 16 * tx.size(), cudaMemcpyHostToDevice, s->st) ||
            cudaMemcpyAsync(s->band_ty, ty.data(), 16 * ty.size(), cudaMemcpyHostToDevice, s->st) ||
            cudaMemcpyAsync(s->band_ox, ox.data(), 4 * ox.size(), cudaMemcpyHostToDevice, s->st) ||
            cudaMemcpyAsync(s->band_oy, oy.data(), 4 * oy.size(), cudaMemcpyHostToDevice, s->st)) {
          r = fail(s, FM_ECUDA, "upload stencil");
          break;
        }
        // the host vectors must outlive the copies
        if (cudaStreamSynchronize(s->st) != cudaSuccess) { r = fail(s, FM_ECUDA, "stencil sync"); break; }
      }
    }
    if (p->protocol == FM_PROJECTIVE_POISSON && (r = poisson_setup(s)) != FM_OK) break;
    // stage the rows in the EE scratch (free until the first entropy call)
    z64* dpx = s->ee_pb;
    z64* dpy = s->ee_pb + s->Lx;
    if (cudaMemcpyAsync(dpx, px.data(), 16 * s->Lx, cudaMemcpyHostToDevice, s->st) ||
        cudaMemcpyAsync(dpy, py.data(), 16 * s->Ly, cudaMemcpyHostToDevice, s->st)) {
      r = fail(s, FM_ECUDA, "upload propagator rows");
      break;
    }
    if (p->precision == FM_FP64) {
      if (expand_propagator_z(s->st, dpx, dpy, s->Lx, s->Ly, s->P) ||
          neel_init_z(s->st, s->U, s->L, s->N, s->B, s->occ_d)) {
        r = fail(s, FM_ECUDA, "init kernels");
        break;
      }
      s->launches += 2;
    } else {
      if (expand_propagator_planes(s->st, dpx, dpy, s->Lx, s->Ly, s->Ah, s->Al) ||
          neel_init_v(s->st, s->V, s->Vh, s->Vl, s->L, s->N, s->B, s->occ_d)) {
        r = fail(s, FM_ECUDA, "init kernels");
        break;
      }
      s->launches += 2;
      MixedCtx& c = s->mc;
      c.st = s->st; c.Lx = s->Lx; c.Ly = s->Ly; c.L = s->L; c.N = s->N; c.B = s->B;
      c.protocol = p->protocol; c.reorth_interval = p->reorth_interval; c.dt = p->dt; c.J = p->J; c.seed = p->seed;
      c.tile_config = p->tile_config;
      c.global_step = 0; c.V = s->V; c.V2 = s->V2; c.Vh = s->Vh; c.Vl = s->Vl; c.Ah = s->Ah; c.Al = s->Al;
      c.Th = s->Th; c.Tl = s->Tl; c.G = s->G; c.R = s->R; c.T = s->T; c.Dinv = s->Dinv; c.X = s->X;
      c.gamma = s->gamma_d; c.traj = s->traj_d; c.step = s->step_d; c.status = s->status_d;
      c.part = s->part_d; c.nocc = s->nocc_d; c.w = s->w_d; c.xbuf = s->xbuf_d; c.vbuf = s->vbuf_d;
      c.log = s->log_d; c.log_count = (int64_t*)s->log_count_d; c.log_capacity = p->event_capacity;
      c.force = s->force_d; c.force_n = 0;
      c.extra = s->mixed_extra; c.launches = 0; c.timer = &s->timer; c.pmw = s->pmw;
      c.prop_banded = 0;
      c.band_tx = s->band_tx; c.band_ty = s->band_ty; c.band_ox = s->band_ox; c.band_oy = s->band_oy;
      c.ntap_x = s->ntap_x; c.ntap_y = s->ntap_y;
      c.rk4buf = (float*)s->rk4buf;
      std::string why2;
      s->mh = mixed_create(&c, &why2);
      if (!s->mh) {
        r = fail(s, FM_ECUDA, "mixed init: " + why2);
        break;
      }
    }
    if (cudaStreamSynchronize(s->st) != cudaSuccess) { r = fail(s, FM_ECUDA, "init sync"); break; }
  } while (0);
  if (r != FM_OK) {
    mixed_free(s->mh);
    delete s;
    return r;
  }
  *out = s;
  return FM_OK;
}

fm_status fm_step(fm_state* s, int32_t nsteps) {
  fm_status r = check_state(s);
  if (r) return r;
  if (nsteps < 0) return fail(s, FM_EINVAL, "nsteps < 0");
  if (nsteps == 0) return FM_OK;
  // once asynchronous entropies exist, the steps run on the high-priority
  // stream, ordered after and before the caller's stream by two events
  cudaStream_t user = s->st;
  const bool bridge = s->hp_st != nullptr;
  if (bridge) {
    CK(cudaEventRecord(s->hp_in, user));
    CK(cudaStreamWaitEvent(s->hp_st, s->hp_in, 0));
    s->st = s->hp_st;
    s->timer.st = s->hp_st;
  }
  r = step_many(s, nsteps);
  if (bridge) {
    s->st = user;
    s->timer.st = user;
    if (s->prm.precision != FM_FP64) s->mc.st = user;
    cudaError_t e = cudaEventRecord(s->hp_out, s->hp_st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, s->hp_out, 0);
    if (e != cudaSuccess && r == FM_OK) r = fail(s, FM_ECUDA, std::string("step stream bridge: ") + cudaGetErrorString(e));
  }
  return r;
}

fm_status fm_set_graphs(fm_state* s, int32_t enable) {
  fm_status r = check_state(s);
  if (r) return r;
  s->graphs_on = enable != 0;
  s->graph_period = 2 * s->prm.reorth_interval;
  return FM_OK;
}

fm_status fm_set_propagation(fm_state* s, int32_t mode) {
  fm_status r = check_state(s);
  if (r) return r;
  if (mode != FM_PROP_DENSE && mode != FM_PROP_BANDED) return fail(s, FM_EINVAL, "unknown propagation mode");
  if (mode == FM_PROP_BANDED && (s->ntap_x == 0 || s->ntap_y == 0))
    return fail(s, FM_EINVAL, "the propagator is too wide for the stencil");
  CK(cudaStreamSynchronize(s->st));
  s->prop_mode = mode;
  if (s->prm.precision != FM_FP64) s->mc.prop_banded = mode == FM_PROP_BANDED;
  s->config_gen += 1;
  if (s->graph_exec) {                 // the captured period used the other propagation
    cudaGraphExecDestroy(s->graph_exec);
    s->graph_exec = nullptr;
  }
  return FM_OK;
}

fm_status fm_force_outcomes(fm_state* s, const fm_event* events, int32_t n) {
  fm_status r = check_state(s);
  if (r) return r;
  if (s->prm.protocol != FM_PROJECTIVE)
    return fail(s, FM_EINVAL, "forced outcomes apply to the fixed-step projective protocol");
  if (n < 0 || (n > 0 && !events)) return fail(s, FM_EINVAL, "bad forced-outcome list");
  if (n > s->prm.event_capacity) return fail(s, FM_EINVAL, "more forced outcomes than event_capacity");
  std::vector<int4> f(n);
  for (int i = 0; i < n; ++i) {
    const fm_event& e = events[i];
    if (e.step < 0 || e.step > 0x7fffffff || e.traj < 0 || e.traj >= s->B || e.site < 0 || e.site >= s->L ||
        (e.outcome != 0 && e.outcome != 1))
      return fail(s, FM_EINVAL, "forced outcome " + std::to_string(i) + " out of range");
    f[i] = make_int4((int)e.step, e.traj, e.site, e.outcome);
  }
  std::sort(f.begin(), f.end(), [](const int4& a, const int4& b) {
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    return a.z < b.z;
  });
  for (int i = 1; i < n; ++i)
    if (f[i].x == f[i - 1].x && f[i].y == f[i - 1].y && f[i].z == f[i - 1].z)
      return fail(s, FM_EINVAL, "a measurement is listed twice");
  CK(cudaStreamSynchronize(s->st));
  if (n > 0) CK(cudaMemcpy(s->force_d, f.data(), sizeof(int4) * (size_t)n, cudaMemcpyHostToDevice));
  s->force_n = n;
  if (s->prm.precision != FM_FP64) s->mc.force_n = n;
  s->config_gen += 1;
  if (s->graph_exec) {                 // the captured period holds the previous list's length
    cudaGraphExecDestroy(s->graph_exec);
    s->graph_exec = nullptr;
  }
  return FM_OK;
}

fm_status fm_set_gammas(fm_state* s, const double* gammas) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!gammas) return fail(s, FM_EINVAL, "gammas is NULL");
  for (int b = 0; b < s->B; ++b)
    if (!(gammas[b] >= 0.0) || !isfinite(gammas[b])) return fail(s, FM_EINVAL, "gamma must be finite, >= 0");
  for (int b = 0; b < s->B; ++b) s->gamma_h[b] = gammas[b];
  // continuous-time protocol: the event times as if the new rates held from t = 0
  if (s->prm.protocol == FM_PROJECTIVE_POISSON)
    for (int b = 0; b < s->B; ++b) poisson_sync(s, b);
  CK(cudaMemcpyAsync(s->gamma_d, s->gamma_h.data(), 8 * s->B, cudaMemcpyHostToDevice, s->st));
  CK(cudaStreamSynchronize(s->st));
  return FM_OK;
}

fm_status fm_reset_trajectory(fm_state* s, int32_t b, uint64_t traj_id, double gamma) {
  fm_status r = check_state(s);
  if (r) return r;
  if (b < 0 || b >= s->B) return fail(s, FM_EINVAL, "trajectory index out of range");
  if (!(gamma >= 0.0) || !isfinite(gamma)) return fail(s, FM_EINVAL, "gamma must be finite, >= 0");
  CK(cudaStreamSynchronize(s->st));
  s->gamma_h[b] = gamma;
  s->traj_h[b] = traj_id;
  s->step_h[b] = 0;
  if (s->prm.protocol == FM_PROJECTIVE_POISSON) poisson_sync(s, b);
  CK(cudaMemcpyAsync(s->gamma_d + b, &s->gamma_h[b], 8, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->traj_d + b, &s->traj_h[b], 8, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemcpyAsync(s->step_d + b, &s->step_h[b], 8, cudaMemcpyHostToDevice, s->st));
  if (s->prm.precision == FM_FP64) {
    CKL(neel_init_z(s->st, s->U + (int64_t)b * s->L * s->N, s->L, s->N, 1, s->occ_d), 1);
  } else {
    const int64_t o = (int64_t)b * 2 * s->L * s->N;
    CKL(neel_init_v(s->st, s->V + o, s->Vh + o, s->Vl + o, s->L, s->N, 1, s->occ_d), 1);
  }
  CK(cudaStreamSynchronize(s->st));
  return FM_OK;
}

fm_status fm_steps_done(fm_state* s, int32_t b, int64_t* out) {
  if (!s || !out) return FM_EINVAL;
  if (b < 0 || b >= s->B) return fail(s, FM_EINVAL, "trajectory index out of range");
  *out = s->step_h[b];
  return FM_OK;
}

fm_status fm_entropy(fm_state* s, int32_t b, const int32_t* sites, int32_t n, double* S_out) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!S_out || b < 0 || b >= s->B) return fail(s, FM_EINVAL, "bad trajectory index or output");
  if ((r = settle(s))) return r;
  r = validate_sites(s, sites, n);
  if (r) return r;
  return entropy_impl(s, b, sites, n, S_out);
}

fm_status fm_entropy_async(fm_state* s, int32_t b, const int32_t* sites, int32_t n, int64_t* ticket) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!ticket || b < 0 || b >= s->B) return fail(s, FM_EINVAL, "bad trajectory index or ticket");
  if ((r = settle(s))) return r;
  r = validate_sites(s, sites, n);
  if (r) return r;
  return entropy_async_impl(s, b, sites, n, ticket);
}

fm_status fm_entropy_ready(fm_state* s, int64_t ticket, int32_t* ready) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!ready || ticket < 0 || ticket >= s->ea_next || ticket < s->ea_next - kAsyncSlots)
    return fail(s, FM_EINVAL, "unknown or expired ticket");
  if ((r = ea_check(s))) return r;
  *ready = 0;
  {
    std::lock_guard<std::mutex> lk(s->ea_mu);
    if (s->ea_issued < ticket + 1) return FM_OK;
  }
  const cudaError_t e = cudaEventQuery(s->ea_done[(int)(ticket % kAsyncSlots)]);
  if (e == cudaSuccess) *ready = 1;
  else if (e != cudaErrorNotReady) return fail(s, FM_ECUDA, std::string("entropy event: ") + cudaGetErrorString(e));
  else (void)cudaGetLastError();
  return FM_OK;
}

fm_status fm_entropy_wait(fm_state* s, int64_t ticket, double* S_out) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!S_out || ticket < 0 || ticket >= s->ea_next || ticket < s->ea_next - kAsyncSlots)
    return fail(s, FM_EINVAL, "unknown or expired ticket");
  const int slot = (int)(ticket % kAsyncSlots);
  ea_wait_issued(s, ticket + 1);
  if ((r = ea_check(s))) return r;
  CK(cudaEventSynchronize(s->ea_done[slot]));
  *S_out = s->ea_host[slot];
  return sync_and_check(s);
}

fm_status fm_set_entropy_method(fm_state* s, int32_t method) {
  fm_status r = check_state(s);
  if (r) return r;
  if (method != FM_EE_FULL && method != FM_EE_SKETCH && method != FM_EE_AUTO)
    return fail(s, FM_EINVAL, "unknown entropy method");
  if (method != FM_EE_FULL && s->prm.precision != FM_MIXED)
    return fail(s, FM_EINVAL, "the entropy sketch needs a mixed-precision state");
  CK(cudaStreamSynchronize(s->st));
  for (int k = 0; k < s->ea_nw; ++k)
    if (s->ea_w[k].st) CK(cudaStreamSynchronize(s->ea_w[k].st));
  s->ee_method = method;
  return FM_OK;
}

fm_status fm_entropy_sketch_info(fm_state* s, int32_t* rank, double* check, int32_t* fell_back) {
  fm_status r = check_state(s);
  if (r) return r;
  if (rank) *rank = s->sk_last_fallback ? 0 : s->sk_last_rank;
  if (check) *check = s->sk_last_chk;
  if (fell_back) *fell_back = s->sk_last_fallback;
  return FM_OK;
}

fm_status fm_density_correlation(fm_state* s, int32_t b, double* c_out) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!c_out || b < 0 || b >= s->B) return fail(s, FM_EINVAL, "bad trajectory index or output");
  if ((r = settle(s))) return r;
  const int L = s->L, N = s->N;
  const int S = std::max(1, L / 2);               // stripe width: the stripe fits the scratch next to U
  double* bins = s->obs;
  BufGuard guard(s, s->st);                       // s->aux
  CK(cudaMemsetAsync(bins, 0, sizeof(double) * L, s->st));
  if (s->prm.precision == FM_FP64) {
    const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
    const z64* U = s->U + (int64_t)b * L * N;
    z64* X = s->aux;                              // L x S stripe of C
    for (int j0 = 0; j0 < L; j0 += S) {
      const int w = std::min(S, L - j0);
      CKL(zgemm<double>(s->st, L, w, N, OP_N, OP_C, one, U, L, 0, U + j0, L, 0, zero, X, L, 0, 1, 0), 1);
      CKL(displacement_bins<double>(s->st, X, L, s->Lx, s->Ly, j0, w, bins), 1);
    }
  } else {
    const c32 one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
    c32* U = (c32*)s->aux;                        // complex64 copy of U_b, then the stripe
    c32* X = U + (int64_t)L * N;
    CKL(v_to_c32(s->st, s->V + (int64_t)b * 2 * L * N, L, N, U), 1);
    for (int j0 = 0; j0 < L; j0 += S) {
      const int w = std::min(S, L - j0);
      CKL(zgemm<float>(s->st, L, w, N, OP_N, OP_C, one, U, L, 0, U + j0, L, 0, zero, X, L, 0, 1, 0), 1);
      CKL(displacement_bins<float>(s->st, X, L, s->Lx, s->Ly, j0, w, bins), 1);
    }
  }
  std::vector<double> h(L);
  CK(cudaMemcpyAsync(h.data(), bins, sizeof(double) * L, cudaMemcpyDeviceToHost, s->st));
  if ((r = sync_and_check(s))) return r;
  for (int d = 0; d < L; ++d) c_out[d] = -h[d] / (double)L;
  return FM_OK;
}

fm_status fm_particle_covariance(fm_state* s, int32_t b, const int32_t* A, int32_t nA, const int32_t* B,
                                 int32_t nB, double* G_out) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!G_out || b < 0 || b >= s->B) return fail(s, FM_EINVAL, "bad trajectory index or output");
  if ((r = settle(s))) return r;
  if ((r = validate_sites(s, A, nA)) || (r = validate_sites(s, B, nB))) return r;
  std::vector<int32_t> AB(A, A + nA);
  AB.insert(AB.end(), B, B + nB);
  if ((r = validate_sites(s, AB.data(), (int32_t)AB.size()))) return fail(s, FM_EINVAL, "A and B overlap");
  if (nA == 0 || nB == 0) { *G_out = 0.0; return FM_OK; }
  const int L = s->L, N = s->N;
  BufGuard guard(s, s->st);                       // s->aux
  CK(cudaMemcpyAsync(s->ee_sites, AB.data(), sizeof(int) * (nA + nB), cudaMemcpyHostToDevice, s->st));
  double* part = s->obs + L;
  double* res = part + abs2_partials();
  if (s->prm.precision == FM_FP64) {
    const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
    z64* rows = s->aux;                           // (nA + nB) x N, ld nA + nB
    CKL(gather_rows_z(s->st, s->U + (int64_t)b * L * N, L, N, s->ee_sites, nA + nB, rows), 1);
    const int ld = nA + nB;
    CKL(zgemm<double>(s->st, nA, nB, N, OP_N, OP_C, one, rows, ld, 0, rows + nA, ld, 0, zero, s->G, nA, 0, 1, 0), 1);
    CKL(sum_abs2<double>(s->st, s->G, (int64_t)nA * nB, part, res), 2);
  } else {
    const c32 one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
    c32* rows = (c32*)s->aux;
    c32* M = (c32*)s->G;
    CKL(gather_rows_c32(s->st, s->V + (int64_t)b * 2 * L * N, L, N, s->ee_sites, nA + nB, rows), 1);
    const int ld = nA + nB;
    CKL(zgemm<float>(s->st, nA, nB, N, OP_N, OP_C, one, rows, ld, 0, rows + nA, ld, 0, zero, M, nA, 0, 1, 0), 1);
    CKL(sum_abs2<float>(s->st, M, (int64_t)nA * nB, part, res), 2);
  }
  CK(cudaMemcpyAsync(G_out, res, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

fm_status fm_mutual_info(fm_state* s, int32_t b, const int32_t* A, int32_t nA, const int32_t* B, int32_t nB,
                         double* I_out) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!I_out || b < 0 || b >= s->B) return fail(s, FM_EINVAL, "bad trajectory index or output");
  if ((r = settle(s))) return r;
  if ((r = validate_sites(s, A, nA)) || (r = validate_sites(s, B, nB))) return r;
  std::vector<int32_t> AB(A, A + nA);
  AB.insert(AB.end(), B, B + nB);
  r = validate_sites(s, AB.data(), (int32_t)AB.size());
  if (r) return fail(s, FM_EINVAL, "A and B overlap");
  std::sort(AB.begin(), AB.end());
  double SA, SB, SAB;
  if ((r = entropy_impl(s, b, A, nA, &SA)) || (r = entropy_impl(s, b, B, nB, &SB)) ||
      (r = entropy_impl(s, b, AB.data(), (int32_t)AB.size(), &SAB)))
    return r;
  *I_out = SA + SB - SAB;
  return FM_OK;
}

fm_status fm_copy_U(fm_state* s, int32_t b, void* host_c128, int64_t ld) {
  fm_status r = check_state(s);
  if (r) return r;
  if (b < 0 || b >= s->B || !host_c128 || ld < s->L) return fail(s, FM_EINVAL, "bad copy_U arguments");
  if ((r = settle(s))) return r;
  const z64* src;
  BufGuard guard(s, s->st);                       // s->aux
  if (s->prm.precision == FM_FP64) src = s->U + (int64_t)b * s->L * s->N;
  else {
    CKL(v_to_z(s->st, s->V + (int64_t)b * 2 * s->L * s->N, s->L, s->N, s->aux), 1);
    src = s->aux;
  }
  CK(cudaMemcpy2DAsync(host_c128, ld * 16, src, (size_t)s->L * 16, (size_t)s->L * 16, s->N,
                       cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

fm_status fm_set_U(fm_state* s, int32_t b, const void* host_c128, int64_t ld) {
  fm_status r = check_state(s);
  if (r) return r;
  if (b < 0 || b >= s->B || !host_c128 || ld < s->L) return fail(s, FM_EINVAL, "bad set_U arguments");
  CK(cudaStreamSynchronize(s->st));
  if (s->prm.precision == FM_FP64) {
    CK(cudaMemcpy2DAsync(s->U + (int64_t)b * s->L * s->N, (size_t)s->L * 16, host_c128, ld * 16,
                         (size_t)s->L * 16, s->N, cudaMemcpyHostToDevice, s->st));
  } else {
    BufGuard guard(s, s->st);                     // s->aux
    CK(cudaMemcpy2DAsync(s->aux, (size_t)s->L * 16, host_c128, ld * 16, (size_t)s->L * 16, s->N,
                         cudaMemcpyHostToDevice, s->st));
    const int64_t o = (int64_t)b * 2 * s->L * s->N;
    CKL(z_to_v(s->st, s->aux, s->L, s->N, s->V + o, s->Vh + o, s->Vl + o), 1);
  }
  return sync_and_check(s);
}

fm_status fm_occupations(fm_state* s, int32_t b, double* host_n) {
  fm_status r = check_state(s);
  if (r) return r;
  if (b < 0 || b >= s->B || !host_n) return fail(s, FM_EINVAL, "bad occupations arguments");
  const int nch = occupation_chunks(s->L, s->N, 1);
  if (s->prm.precision == FM_FP64) {
    CKL(rownorm_partials_z(s->st, s->U + (int64_t)b * s->L * s->N, s->L, s->N, 1, s->part_d, nch), 1);
  } else {
    CKL(rownorm_partials_v(s->st, s->V + (int64_t)b * 2 * s->L * s->N, s->L, s->N, 1, s->part_d, nch), 1);
  }
  CKL(reduce_occupations(s->st, s->part_d, nch, s->L, 1, s->nocc_d, nullptr, s->gamma_d, s->prm.dt, s->traj_d,
                         s->step_d, s->prm.seed), 1);
  CK(cudaMemcpyAsync(host_n, s->nocc_d, 8 * s->L, cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

fm_status fm_orthonormality_error(fm_state* s, int32_t b, const int32_t* cols, int32_t ncols, double* err) {
  fm_status r = check_state(s);
  if (r) return r;
  if (b < 0 || b >= s->B || !err || ncols < 1 || ncols > std::min(s->N, 64) || !cols)
    return fail(s, FM_EINVAL, "bad orthonormality arguments (1 <= ncols <= min(N, 64))");
  for (int i = 0; i < ncols; ++i)
    if (cols[i] < 0 || cols[i] >= s->N) return fail(s, FM_EINVAL, "column index out of range");
  const int L = s->L, N = s->N;
  // aux <- U_b as complex128 (L x N), then Gs = U[:, cols]^dag U (ncols x N) in R
  const z64* U;
  BufGuard guard(s, s->st);                       // s->aux
  if (s->prm.precision == FM_FP64) U = s->U + (int64_t)b * L * N;
  else {
    CKL(v_to_z(s->st, s->V + (int64_t)b * 2 * L * N, L, N, s->aux), 1);
    U = s->aux;
  }
  z64* Uc = s->chk_cols;
  for (int i = 0; i < ncols; ++i)
    CK(cudaMemcpyAsync(Uc + (int64_t)i * L, U + (int64_t)cols[i] * L, 16 * L, cudaMemcpyDeviceToDevice, s->st));
  const z64 one = {1.0, 0.0}, zero = {0.0, 0.0};
  CKL(zgemm<double>(s->st, ncols, N, L, OP_C, OP_N, one, Uc, L, 0, U, L, 0, zero, s->chk_G, ncols, 0, 1, 0), 1);
  CK(cudaMemcpyAsync(s->ee_sites, cols, 4 * ncols, cudaMemcpyHostToDevice, s->st));
  CK(cudaMemsetAsync(s->ee_max, 0, 8, s->st));
  CKL(max_abs_minus_identity(s->st, s->chk_G, ncols, N, s->ee_sites, s->ee_max), 1);
  CK(cudaMemcpyAsync(err, s->ee_max, 8, cudaMemcpyDeviceToHost, s->st));
  return sync_and_check(s);
}

fm_status fm_take_events(fm_state* s, fm_event* out, int32_t cap, int32_t* count, int64_t* dropped) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!count || !dropped || cap < 0 || (cap > 0 && !out)) return fail(s, FM_EINVAL, "bad take_events arguments");
  CK(cudaStreamSynchronize(s->st));
  unsigned long long n = 0;
  CK(cudaMemcpy(&n, s->log_count_d, 8, cudaMemcpyDeviceToHost));
  const int64_t have = std::min<int64_t>((int64_t)n, s->prm.event_capacity);
  const int64_t take = std::min<int64_t>(have, cap);
  if (take > 0) CK(cudaMemcpy(out, s->log_d, take * sizeof(fm_event), cudaMemcpyDeviceToHost));
  *count = (int32_t)take;
  *dropped = (int64_t)n - take;
  CK(cudaMemset(s->log_count_d, 0, 8));
  return FM_OK;
}

fm_status fm_save(fm_state* s, const char* path) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!path) return fail(s, FM_EINVAL, "path is NULL");
  CK(cudaStreamSynchronize(s->st));
  const size_t ubytes = (s->prm.precision == FM_FP64) ? (size_t)s->B * s->L * s->N * 16
                                                       : (size_t)s->B * 2 * s->L * s->N * 4;
  std::vector<char> host(ubytes);
  CK(cudaMemcpy(host.data(), s->prm.precision == FM_FP64 ? (void*)s->U : (void*)s->V, ubytes,
                cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(s, FM_EINVAL, std::string("cannot open ") + path);
  const char magic[8] = {'F', 'M', 'C', 'K', 'P', 'T', '0', '1'};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(&s->prm, sizeof(fm_params), 1, f) == 1 &&
            fwrite(&s->global_steps, 8, 1, f) == 1 && fwrite(s->gamma_h.data(), 8, s->B, f) == (size_t)s->B &&
            fwrite(s->traj_h.data(), 8, s->B, f) == (size_t)s->B &&
            fwrite(s->step_h.data(), 8, s->B, f) == (size_t)s->B && fwrite(host.data(), 1, ubytes, f) == ubytes;
  fclose(f);
  if (!ok) return fail(s, FM_EINVAL, "short write");
  return FM_OK;
}

fm_status fm_load(fm_state* s, const char* path) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!path) return fail(s, FM_EINVAL, "path is NULL");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(s, FM_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  fm_params p;
  int64_t gsteps;
  std::vector<double> g(s->B);
  std::vector<uint64_t> t(s->B);
  std::vector<int64_t> st(s->B);
  const size_t ubytes = (s->prm.precision == FM_FP64) ? (size_t)s->B * s->L * s->N * 16
                                                       : (size_t)s->B * 2 * s->L * s->N * 4;
  std::vector<char> host(ubytes);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "FMCKPT01", 8) == 0 &&
            fread(&p, sizeof(fm_params), 1, f) == 1 && fread(&gsteps, 8, 1, f) == 1 &&
            fread(g.data(), 8, s->B, f) == (size_t)s->B && fread(t.data(), 8, s->B, f) == (size_t)s->B &&
            fread(st.data(), 8, s->B, f) == (size_t)s->B && fread(host.data(), 1, ubytes, f) == ubytes;
  fclose(f);
  if (!ok) return fail(s, FM_EINVAL, "bad or truncated checkpoint");
  if (p.Lx != s->prm.Lx || p.Ly != s->prm.Ly || p.batch != s->prm.batch || p.precision != s->prm.precision ||
      p.protocol != s->prm.protocol || p.seed != s->prm.seed || p.dt != s->prm.dt || p.J != s->prm.J)
    return fail(s, FM_EINVAL, "checkpoint does not match this state's parameters");
  CK(cudaStreamSynchronize(s->st));
  s->gamma_h = g; s->traj_h = t; s->step_h = st; s->global_steps = gsteps;
  s->settled_step = -1;
  if (s->prm.protocol == FM_PROJECTIVE_POISSON)
    for (int b = 0; b < s->B; ++b) poisson_sync(s, b);
  CK(cudaMemcpy(s->gamma_d, g.data(), 8 * s->B, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->traj_d, t.data(), 8 * s->B, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->step_d, st.data(), 8 * s->B, cudaMemcpyHostToDevice));
  if (s->prm.precision == FM_FP64) {
    CK(cudaMemcpy(s->U, host.data(), ubytes, cudaMemcpyHostToDevice));
  } else {
    CK(cudaMemcpy(s->V, host.data(), ubytes, cudaMemcpyHostToDevice));
    CKL(split_planes(s->st, s->V, s->Vh, s->Vl, (int64_t)s->B * 2 * s->L * s->N), 1);
  }
  return sync_and_check(s);
}

fm_status fm_set_timing(fm_state* s, int32_t enable) {
  fm_status r = check_state(s);
  if (r) return r;
  CK(cudaStreamSynchronize(s->st));
  s->timer.on = enable != 0;
  return FM_OK;
}

fm_status fm_phase_times(fm_state* s, double* ms, int64_t* counts) {
  fm_status r = check_state(s);
  if (r) return r;
  if (!s->timer.collect(ms, counts)) return fail(s, FM_ECUDA, "event timing failed");
  return FM_OK;
}

fm_status fm_reorth_stats(fm_state* s, int64_t* checks, int64_t* extra_passes, double* maxima) {
  fm_status r = check_state(s);
  if (r) return r;
  int64_t cnt[2] = {0, 0};
  double mx[4] = {0.0, 0.0, 0.0, 0.0};
  if (s->mh) {
    if (mixed_guard_stats(s->mh, s->st, cnt, mx) != FM_OK) return fail(s, FM_ECUDA, "guard statistics readback");
  }
  if (checks) *checks = cnt[0];
  if (extra_passes) *extra_passes = cnt[1];
  if (maxima)
    for (int i = 0; i < 4; ++i) maxima[i] = mx[i];
  return FM_OK;
}

extern "C" int fmx_poisson_draw(unsigned long long seed, unsigned long long traj, long long e, int L, double* out) {
  if (!out || L < 1 || e < 0) return -1;
  const PoisDraw d = poisson_draw(seed, traj, e, L);
  out[0] = d.u_wait;
  out[1] = d.site;
  out[2] = d.u;
  return 0;
}

extern "C" int fmx_poisson_taps(int n, int w, double J, double tau, double* out) {
  if (!out || n < 1 || w > 4 * kBandMaxTaps || !std::isfinite(J) || !(tau >= 0.0)) return -1;
  if (w >= 0 && 2 * w + 1 > n) return -1;
  poisson_taps(n, w, J, tau, (z64*)out);
  return 0;
}

extern "C" int fmx_poisson_width(int n, double J, double dt) {
  if (n < 1 || !std::isfinite(J) || !(dt >= 0.0)) return -2;
  return poisson_width(n, J, dt);
}

fm_status fm_autotune(const fm_params* p, void* d_workspace, size_t ws_bytes, void* cuda_stream, int32_t steps,
                      int32_t max_reorth, double ortho_tol, int32_t use_graphs, fm_tuning* out) {
  if (!p || !out || steps < 1 || max_reorth < 1 || !(ortho_tol > 0.0)) return FM_EINVAL;
  fm_params p0 = *p;
  p0.tile_config = 0;
  p0.reorth_interval = 1;
  fm_state* s = nullptr;
  fm_status r = fm_init_state(&p0, d_workspace, ws_bytes, cuda_stream, &s);
  if (r) return r;
  const bool mixed = p->precision == FM_MIXED;
  std::vector<int> tiles;
  if (mixed) {
    for (int bn : {1, 2}) {
      if (bn == 2 && s->N % 256) continue;
      for (int g : {2, 3, 4}) tiles.push_back(bn | (g << 2));
    }
  } else {
    tiles.push_back(0);
  }
  std::vector<int> cols;
  for (int i = 0; i < std::min(s->N, 64); ++i) cols.push_back((int)((int64_t)i * s->N / std::min(s->N, 64)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fm_tuning best{0, 1, 0.0, 0.0, 0, 0, 0.0}, best1{0, 1, 0.0, 0.0, 0, 0, 0.0};
  bool have = false, have1 = false;
  int tried = 0, rejected = 0;
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { r = FM_ECUDA; break; }
    // candidates: every tile configuration x interval, then (mixed precision, interval > 1)
    // the drain intervals of the first-pass product for the fastest accepted one, then
    // (batches of three or more) the fastest with one Cholesky chain per trajectory
    std::vector<std::pair<int, int>> cands;
    int stage = 0;
    for (int k = 1; k <= max_reorth; k *= 2)
      for (int tc : tiles) cands.push_back({tc, k});
    for (size_t ci = 0; ci < cands.size() && r == FM_OK; ++ci) {
        const int tc = cands[ci].first, k = cands[ci].second;
        if ((r = retune(s, tc, k))) break;
        if ((r = fm_set_graphs(s, use_graphs ? 1 : 0))) break;
        const int period = 2 * k;
        const int nt = ((steps + period - 1) / period) * period;
        if ((r = fm_step(s, period))) break;                     // warm-up (and graph capture)
        if (cudaEventRecord(e0, s->st) != cudaSuccess) { r = fail(s, FM_ECUDA, "event"); break; }
        if ((r = fm_step(s, nt))) break;
        if (cudaEventRecord(e1, s->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          r = fail(s, FM_ECUDA, "event");
          break;
        }
        if ((r = sync_and_check(s))) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        // orthonormality after each of 2k single steps: at the period ends (after a second
        // pass) against ortho_tol; in between (first pass only; observables settle such a
        // state first, fm_entropy etc.) against 100 ortho_tol, where the next step's
        // occupations, the only other reader, move by <= 1e-4 relative
        double worst = 0.0, worst_mid = 0.0;
        for (int i = 0; i < period && r == FM_OK; ++i) {
          if ((r = fm_step(s, 1))) break;
          const bool end = s->global_steps % k == 0;
          for (int b : {0, s->B - 1}) {
            double e = 0.0;
            if ((r = fm_orthonormality_error(s, b, cols.data(), (int)cols.size(), &e))) break;
            if (end) worst = std::max(worst, e);
            else worst_mid = std::max(worst_mid, e);
          }
        }
        if (r) break;
        fm_tuning cand{tc, k, (double)ms / nt, worst, 0, 0, worst_mid};
        ++tried;
        if (k == 1 && (!have1 || cand.ms_per_step < best1.ms_per_step)) { best1 = cand; have1 = true; }
        if (worst <= ortho_tol && worst_mid <= 100.0 * ortho_tol) {
          if (!have || cand.ms_per_step < best.ms_per_step) { best = cand; have = true; }
        } else {
          ++rejected;
        }
        if (ci + 1 == cands.size() && mixed && have) {
          if (stage == 0) {
            stage = 1;
            if (best.reorth_interval > 1 && !(best.tile_config >> 5))
              for (int d = 1; d <= 2; ++d) cands.push_back({best.tile_config | (d << 5), best.reorth_interval});
          }
          if (stage == 1 && ci + 1 == cands.size()) {
            stage = 2;
            if (s->B >= 3) cands.push_back({best.tile_config | FM_TILE_CHOL_CHAINS, best.reorth_interval});
          }
        }
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  fm_destroy(s);
  if (r) return r;
  *out = have ? best : best1;
  out->tried = tried;
  out->rejected = rejected;
  return FM_OK;
}

// ------------------------------------------------------------------ several states in one graph
struct fm_group {
  std::vector<fm_state*> s;
  cudaStream_t st = nullptr;            // the caller's stream the graph replays on
  cudaStream_t origin = nullptr;        // capture origin
  std::vector<cudaStream_t> br;         // one capture branch per state
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join, in;
  cudaGraphExec_t exec = nullptr;
  int period = 0;
  std::vector<int64_t> per;             // launches of one period, per state
  std::vector<int64_t> gen;             // config_gen of each state at capture
  std::string err;
};

namespace {
int64_t gcd64(int64_t a, int64_t b) { return b ? gcd64(b, a % b) : a; }

void group_release(fm_group* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  g->exec = nullptr;
  for (cudaStream_t b : g->br)
    if (b) cudaStreamDestroy(b);
  g->br.clear();
  if (g->origin) cudaStreamDestroy(g->origin);
  for (cudaEvent_t e : g->join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : g->in)
    if (e) cudaEventDestroy(e);
  g->join.clear();
  g->in.clear();
  if (g->fork) cudaEventDestroy(g->fork);
  if (g->done) cudaEventDestroy(g->done);
}

// One period of every state, each on its own branch of one graph (forked from the origin
// stream, joined back into it), so that the states' kernels overlap on the device.
fm_status group_capture(fm_group* g) {
  if (g->exec) {
    cudaGraphExecDestroy(g->exec);
    g->exec = nullptr;
  }
  for (fm_state* s : g->s)
    if (cudaStreamSynchronize(s->st) != cudaSuccess) return FM_ECUDA;
  cudaGraph_t graph = nullptr;
  fm_status r = FM_OK;
  if (cudaStreamBeginCapture(g->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FM_ECUDA;
  cudaError_t e = cudaEventRecord(g->fork, g->origin);
  for (size_t i = 0; i < g->s.size() && r == FM_OK && e == cudaSuccess; ++i) {
    e = cudaStreamWaitEvent(g->br[i], g->fork, 0);
    if (e == cudaSuccess) r = issue_period(g->s[i], g->br[i], g->period, &g->per[i]);
    if (r == FM_OK && e == cudaSuccess) e = cudaEventRecord(g->join[i], g->br[i]);
    if (r == FM_OK && e == cudaSuccess) e = cudaStreamWaitEvent(g->origin, g->join[i], 0);
  }
  const cudaError_t e2 = cudaStreamEndCapture(g->origin, &graph);
  if (r == FM_OK && (e != cudaSuccess || e2 != cudaSuccess)) {
    g->err = std::string("group capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2);
    r = FM_ECUDA;
  } else if (r != FM_OK) {
    g->err = "group capture: a state failed (see its fm_last_error)";
  }
  if (r == FM_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) {
    g->err = "group graph instantiation";
    r = FM_ECUDA;
  }
  if (graph) cudaGraphDestroy(graph);
  for (size_t i = 0; i < g->s.size(); ++i) g->gen[i] = g->s[i]->config_gen;
  return r;
}
}  // namespace

fm_status fm_group_create(fm_state* const* states, int32_t n, void* cuda_stream, fm_group** out) {
  if (!out || !states || n < 1 || n > 4096) return FM_EINVAL;
  *out = nullptr;
  int64_t P = 1;
  for (int i = 0; i < n; ++i) {
    fm_state* s = states[i];
    if (!s || check_state(s) != FM_OK || !graph_capable(s)) return FM_EINVAL;
    for (int j = 0; j < i; ++j)
      if (states[j] == s) return FM_EINVAL;
    const int64_t q = 2 * (int64_t)s->prm.reorth_interval;
    P = P / gcd64(P, q) * q;
    if (P > 256) return FM_EINVAL;
  }
  fm_group* g = new fm_group();
  g->s.assign(states, states + n);
  g->st = (cudaStream_t)cuda_stream;
  g->period = (int)P;
  g->per.assign(n, 0);
  g->gen.assign(n, -1);
  bool ok = cudaStreamCreateWithFlags(&g->origin, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) == cudaSuccess;
  g->br.assign(n, nullptr);
  g->join.assign(n, nullptr);
  g->in.assign(n, nullptr);
  for (int i = 0; i < n && ok; ++i)
    ok = cudaStreamCreateWithFlags(&g->br[i], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->join[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&g->in[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    group_release(g);
    delete g;
    return FM_ECUDA;
  }
  *out = g;
  return FM_OK;
}

fm_status fm_group_step(fm_group* g, int32_t nsteps) {
  if (!g) return FM_EINVAL;
  if (nsteps < 0 || nsteps % g->period) {
    g->err = "nsteps must be a multiple of the group period " + std::to_string(g->period);
    return FM_EINVAL;
  }
  for (fm_state* s : g->s) {
    if (check_state(s) != FM_OK) {
      g->err = "a state holds an error";
      return FM_ESTATE;
    }
    if (s->global_steps % g->period) {
      g->err = "every state must stand at a multiple of the group period";
      return FM_EINVAL;
    }
  }
  if (nsteps == 0) return FM_OK;
  bool stale = !g->exec;
  for (size_t i = 0; i < g->s.size(); ++i) stale |= g->gen[i] != g->s[i]->config_gen;
  if (stale) {
    const fm_status r = group_capture(g);
    if (r) return r;
  }
  // the caller's stream waits for every state's stream, replays, and every state's stream
  // then waits for it (so later calls on a state see the steps)
  for (size_t i = 0; i < g->s.size(); ++i)
    if (cudaEventRecord(g->in[i], g->s[i]->st) != cudaSuccess || cudaStreamWaitEvent(g->st, g->in[i], 0) != cudaSuccess)
      return FM_ECUDA;
  const int reps = nsteps / g->period;
  for (int k = 0; k < reps; ++k)
    if (cudaGraphLaunch(g->exec, g->st) != cudaSuccess) {
      g->err = "cudaGraphLaunch";
      return FM_ECUDA;
    }
  if (cudaEventRecord(g->done, g->st) != cudaSuccess) return FM_ECUDA;
  for (size_t i = 0; i < g->s.size(); ++i) {
    fm_state* s = g->s[i];
    if (cudaStreamWaitEvent(s->st, g->done, 0) != cudaSuccess) return FM_ECUDA;
    s->global_steps += nsteps;
    for (int b = 0; b < s->B; ++b) s->step_h[b] += nsteps;
    s->launches += reps * g->per[i];
  }
  return FM_OK;
}

int32_t fm_group_period(const fm_group* g) { return g ? g->period : 0; }

const char* fm_group_last_error(const fm_group* g) { return g ? g->err.c_str() : "null group"; }

void fm_group_destroy(fm_group* g) {
  if (!g) return;
  if (g->st) cudaStreamSynchronize(g->st);
  group_release(g);
  delete g;
}

int64_t fm_kernel_launches(const fm_state* s) { return s ? s->launches + s->ea_launches.load() : 0; }

const char* fm_last_error(const fm_state* s) { return s ? s->err.c_str() : "null state"; }

void fm_destroy(fm_state* s) {
  if (!s) return;
  if (s->ea_st) {
    {
      std::lock_guard<std::mutex> lk(s->ea_mu);
      s->ea_stop = true;
    }
    s->ea_cv.notify_all();
    for (int k = 0; k < s->ea_nw; ++k)
      if (s->ea_w[k].th.joinable()) s->ea_w[k].th.join();   // the threads drain the queue first
    for (int k = 0; k < s->ea_nw; ++k)
      if (s->ea_w[k].st) {
        cudaStreamSynchronize(s->ea_w[k].st);
        cudaStreamDestroy(s->ea_w[k].st);
      }
    cudaStreamSynchronize(s->hp_st);
    cudaStreamDestroy(s->hp_st);
    cudaEventDestroy(s->hp_in);
    cudaEventDestroy(s->hp_out);
    for (int i = 0; i < s->ea_ring; ++i) {
      cudaEventDestroy(s->ea_M_ready[i]);
      cudaEventDestroy(s->ea_M_free[i]);
    }
    for (int i = 0; i < kAsyncSlots; ++i) cudaEventDestroy(s->ea_done[i]);
    cudaFreeHost(s->ea_host);
  }
  if (s->ee_buf_ev) cudaEventDestroy(s->ee_buf_ev);
  if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  mixed_free(s->mh);
  delete s;
}

}  // extern "C"
