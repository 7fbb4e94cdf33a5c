// Structured propagation: U <- exp(-i H~ dt) U as a stencil.
//
// The ring's propagator is circulant, P_ab = p_{(a - b) mod L} with
// p_r = (1/L) sum_k e^{i k r} e^{-2 i J dt cos k} (App. A), and its entries fall
// off like Bessel functions, |p_r| ~ |J_r(2 J dt)|: below 1e-15 beyond r = 8 at
// dt = 0.05.  The torus propagator is P_x (x) P_y.  So P U is a stencil along
// x (then along y) over the taps above 1e-15 -- the same product as the dense
// GEMM up to those dropped entries, for one read and one write of U per
// direction instead of L^2 N multiply-adds.  Offsets and taps come from the
// host; tiny lattices keep every tap.
#include "kernels.h"

namespace fm {

template <typename T, int LAYOUT>
struct band_io;
template <typename T>
struct band_io<T, 0> {  // complex128 U, L x N per trajectory
  FM_DEVFN static cplx<T> ld(const void* base, int64_t b, int L, int N, int i, int k) {
    const z64 z = ((const z64*)base)[b * L * (int64_t)N + i + (int64_t)k * L];
    return cmk<T>((T)z.re, (T)z.im);
  }
  FM_DEVFN static void st(void* base, int64_t b, int L, int N, int i, int k, cplx<T> v) {
    ((z64*)base)[b * L * (int64_t)N + i + (int64_t)k * L] = cmk((double)v.re, (double)v.im);
  }
};
template <typename T>
struct band_io<T, 1> {  // float V, 2L x N per trajectory (column k = [Re; Im])
  FM_DEVFN static cplx<T> ld(const void* base, int64_t b, int L, int N, int i, int k) {
    const float* V = (const float*)base + b * 2 * L * (int64_t)N + (int64_t)k * 2 * L;
    return cmk<T>((T)V[i], (T)V[L + i]);
  }
  FM_DEVFN static void st(void* base, int64_t b, int L, int N, int i, int k, cplx<T> v) {
    float* V = (float*)base + b * 2 * L * (int64_t)N + (int64_t)k * 2 * L;
    V[i] = (float)v.re;
    V[L + i] = (float)v.im;
  }
};

// out[i, k] = sum_t taps[t] in[site i shifted back by off[t] along dir, k].  The
// offsets are consecutive (off[t] = off[0] + t), so the sources of a run of
// outputs along dir are one contiguous (periodic) run of inputs: each block
// stages that run plus the stencil's halo in shared memory (coalesced loads),
// then every thread sums its taps from shared memory.
//   dir 0 (x, unit stride): a block covers 256 consecutive x of one row y and
//     kBandCols columns per stage.
//   dir 1 (y, stride Lx): a block covers 32 consecutive x (one per lane) and 64
//     (float) or 32 (double) consecutive y, one column per stage.
// blockIdx.y picks a chunk of columns, blockIdx.z the trajectory; with
// `partial`, the row sums of |out|^2 over the chunk go to partial[(b nch + chunk) L + i].
constexpr int kBandSegX = 256;
constexpr int kBandCols = 8;
constexpr int seg_y(int layout) { return layout == 0 ? 32 : 64; }

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(256) band_x_kernel(const void* __restrict__ in, void* out, int L, int N, int Lx,
                                                     const z64* __restrict__ taps, const int* __restrict__ off,
                                                     int ntap, int per, double* partial, int nch, int tap_stride) {
  constexpr int W = kBandSegX + kBandMaxTaps - 1;
  __shared__ cplx<T> buf[kBandCols][W];
  __shared__ cplx<T> tp[kBandMaxTaps];
  const int64_t b = blockIdx.z;
  taps += b * tap_stride;
  const int tid = threadIdx.x;
  if (tid < ntap) tp[tid] = cmk<T>((T)taps[tid].re, (T)taps[tid].im);
  const int nseg = (Lx + kBandSegX - 1) / kBandSegX;
  const int seg = blockIdx.x % nseg, y = blockIdx.x / nseg;
  const int p0 = seg * kBandSegX;
  const int offmax = off[0] + ntap - 1;
  const int w = kBandSegX + ntap - 1;               // staged inputs per column
  const int pos = p0 + tid;
  const int i = pos + Lx * y;
  const int c = blockIdx.y;
  const int k0 = c * per, k1 = min(N, k0 + per);
  double s = 0.0;
  // the staged run of one column holds w <= kBandSegX + kBandMaxTaps - 1 < 2 x 256 inputs:
  // two per thread, all of a stage loaded into registers before any is stored
  int srcq[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int src = (p0 - offmax + tid + 256 * h) % Lx;
    srcq[h] = (src < 0 ? src + Lx : src) + Lx * y;
  }
  for (int kb = k0; kb < k1; kb += kBandCols) {
    const int nk = min(kBandCols, k1 - kb);
    cplx<T> v[kBandCols][2];
#pragma unroll
    for (int kk = 0; kk < kBandCols; ++kk)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (kk < nk && tid + 256 * h < w) v[kk][h] = band_io<T, LAYOUT>::ld(in, b, L, N, srcq[h], kb + kk);
    __syncthreads();                                 // previous stage consumed (and tp written)
#pragma unroll
    for (int kk = 0; kk < kBandCols; ++kk)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        if (kk < nk && tid + 256 * h < w) buf[kk][tid + 256 * h] = v[kk][h];
    __syncthreads();
    if (pos < Lx)
      for (int kk = 0; kk < nk; ++kk) {
        cplx<T> acc = cmk<T>((T)0, (T)0);
        const cplx<T>* src = &buf[kk][tid + ntap - 1];
        for (int t = 0; t < ntap; ++t) {
          const cplx<T> u = src[-t];
          acc.re += tp[t].re * u.re - tp[t].im * u.im;
          acc.im += tp[t].re * u.im + tp[t].im * u.re;
        }
        band_io<T, LAYOUT>::st(out, b, L, N, i, kb + kk, acc);
        if (partial) s += (double)(acc.re * acc.re + acc.im * acc.im);
      }
  }
  if (partial && pos < Lx) partial[(b * nch + c) * L + i] = s;
}

// The x stencil of the float state (mixed precision), 4 consecutive sites per thread.
// A block stages, for kB4Cols columns at a time, the input runs of RB rows (one row
// segment of S = min(Lx, 1024) sites plus the stencil's halo each; RB = 256 / (S / 4)
// rows when rows are short, as on the torus) in shared memory as separate Re and Im
// arrays; each thread then slides a 4-wide window down its run, one new input per tap,
// so a tap costs 2 shared loads and 16 FMAs for 4 outputs (the generic kernel above
// spends 2 complex loads per output and tap).  Outputs go out as float4 where the 4 sites
// are consecutive and aligned.  Grid (segments per row x row groups, column chunks, B).
constexpr int kB4Seg = 1024;
constexpr int kB4Cols = 2;
constexpr int kB4Cap = 1344;                       // staged floats per column and plane
constexpr int kB4Loads = (kB4Cap + 255) / 256;
// staged rows are runp = run rounded up to 4 floats apart, so that each thread's window (which
// starts at its first output's site minus the stencil's reach) is 16-byte aligned and loads as
// float4s: 8 lanes then read 128 contiguous bytes, conflict-free
constexpr int kB4Pad = kB4Cap + 3 * 8;

struct B4Shape {
  int S, tpr, RB, segs, groups;
};
inline B4Shape band4_shape(int Lx, int Ly) {
  B4Shape g;
  g.S = Lx < kB4Seg ? Lx : kB4Seg;
  g.tpr = (g.S + 3) / 4;
  g.RB = 256 / g.tpr;
  if (g.RB < 1) g.RB = 1;
  if (g.RB > Ly) g.RB = Ly;
  g.segs = (Lx + g.S - 1) / g.S;
  g.groups = (Ly + g.RB - 1) / g.RB;
  return g;
}

// NT > 0: a stencil of exactly NT taps (the ring's and the torus's at dt = 0.05 keep 15), with
// the taps in registers and each thread's NT + 3 window inputs loaded once per column, so the
// inner loop is NT x 16 FMAs with static indices; NT = 0: any tap count, a window sliding one
// input per tap.
template <int NT>
__global__ void __launch_bounds__(256, 2) band_x4_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                         int L, int N, int Lx, int Ly, int S, int tpr, int RB, int segs,
                                                         const z64* __restrict__ taps, const int* __restrict__ off,
                                                         int ntap, int per, double* partial, int nch, int tap_stride) {
  __shared__ __align__(16) float sre[kB4Cols][kB4Pad];
  __shared__ __align__(16) float sim[kB4Cols][kB4Pad];
  __shared__ float tre[kBandMaxTaps], tim[kBandMaxTaps];
  const int64_t b = blockIdx.z;
  taps += b * tap_stride;
  const int tid = threadIdx.x;
  if (tid < ntap) {
    tre[tid] = (float)taps[tid].re;
    tim[tid] = (float)taps[tid].im;
  }
  const int seg = blockIdx.x % segs, rg = blockIdx.x / segs;
  const int x0 = seg * S;
  const int run = S + ntap - 1;                    // staged inputs per row
  const int runp = (run + 3) & ~3;                 // their row pitch in shared memory
  const int offmax = off[0] + ntap - 1;
  const int tot = RB * run;
  const int64_t L2 = 2 * (int64_t)L;
  const float* inb = in + b * L2 * N;
  float* outb = out + b * L2 * N;
  // source sites of this thread's staged elements (the same for every column)
  int src[kB4Loads], dst[kB4Loads];
#pragma unroll
  for (int u = 0; u < kB4Loads; ++u) {
    const int q = tid + 256 * u;
    src[u] = -1;
    dst[u] = 0;
    if (q < tot) {
      const int r = q / run, e = q - r * run, y = rg * RB + r;
      dst[u] = r * runp + e;
      if (y < Ly) {
        int x = (x0 - offmax + e) % Lx;
        if (x < 0) x += Lx;
        src[u] = x + Lx * y;
      }
    }
  }
  // this thread's outputs: row r, sites x0 + 4 g .. x0 + 4 g + 3 of it
  const int r = tid / tpr, g = tid - r * tpr, y = rg * RB + r;
  const int xs = x0 + 4 * g;
  const int nval = (r < RB && y < Ly) ? max(0, min(4, min(x0 + S, Lx) - xs)) : 0;
  const int site0 = xs + Lx * y;
  const bool vec = nval == 4 && (site0 % 4) == 0 && (L % 4) == 0;
  const int base = r * runp + 4 * g + ntap - 1;    // staged index of the input for output 0 at tap 0
  const int c = blockIdx.y;
  const int k0 = c * per, k1 = min(N, k0 + per);
  // row sums of |out|^2: float over up to 16 columns, then into double (GB300's FP64 rate is
  // ~1/60 of FP32: a double add per output bounded the whole pass)
  double acc2[4] = {0.0, 0.0, 0.0, 0.0};
  float accf[4] = {0.f, 0.f, 0.f, 0.f};
  int nacc = 0;
  // software pipeline: the next stage's columns are loaded into registers while the current
  // stage is computed from shared memory
  float vr[kB4Cols][kB4Loads], vi[kB4Cols][kB4Loads];
  auto load_stage = [&](int kb) {
    const int nk = min(kB4Cols, k1 - kb);
#pragma unroll
    for (int kk = 0; kk < kB4Cols; ++kk)
#pragma unroll
      for (int u = 0; u < kB4Loads; ++u)
        if (kk < nk && src[u] >= 0) {
          const float* col = inb + (int64_t)(kb + kk) * L2;
          vr[kk][u] = __ldg(col + src[u]);
          vi[kk][u] = __ldg(col + L + src[u]);
        }
  };
  auto store_stage = [&](int kb) {
    const int nk = min(kB4Cols, k1 - kb);
#pragma unroll
    for (int kk = 0; kk < kB4Cols; ++kk)
#pragma unroll
      for (int u = 0; u < kB4Loads; ++u)
        if (kk < nk && src[u] >= 0) {
          sre[kk][dst[u]] = vr[kk][u];
          sim[kk][dst[u]] = vi[kk][u];
        }
  };
  if (k0 < k1) {
    load_stage(k0);
    __syncthreads();                               // the taps are in shared memory
    store_stage(k0);
    __syncthreads();
  }
  float treg[NT > 0 ? NT : 1], timg[NT > 0 ? NT : 1];
#pragma unroll
  for (int t = 0; t < (NT > 0 ? NT : 1); ++t) {
    treg[t] = NT > 0 ? tre[t] : 0.f;
    timg[t] = NT > 0 ? tim[t] : 0.f;
  }
  for (int kb = k0; kb < k1; kb += kB4Cols) {
    const int nk = min(kB4Cols, k1 - kb);
    const bool more = kb + kB4Cols < k1;
    if (more) load_stage(kb + kB4Cols);
    if (NT > 0 && nval == 4) {
      for (int kk = 0; kk < nk; ++kk) {
        const float* ar = sre[kk];
        const float* ai = sim[kk];
        // x[q] = input base - (NT - 1) + q (a 16-byte aligned run: base - (NT - 1) = r runp + 4 g);
        // output e at tap t reads x[NT - 1 + e - t]
        constexpr int NV = (NT + 3 + 3) / 4;
        float xr[4 * NV], xi[4 * NV];
        const float4* wr4 = (const float4*)(ar + base - (NT - 1));
        const float4* wi4 = (const float4*)(ai + base - (NT - 1));
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const float4 a = wr4[v], bb = wi4[v];
          xr[4 * v] = a.x; xr[4 * v + 1] = a.y; xr[4 * v + 2] = a.z; xr[4 * v + 3] = a.w;
          xi[4 * v] = bb.x; xi[4 * v + 1] = bb.y; xi[4 * v + 2] = bb.z; xi[4 * v + 3] = bb.w;
        }
        float orr[4] = {0.f, 0.f, 0.f, 0.f}, oii[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float ur = xr[NT - 1 + e - t], ui = xi[NT - 1 + e - t];
            orr[e] = fmaf(treg[t], ur, orr[e]);
            orr[e] = fmaf(-timg[t], ui, orr[e]);
            oii[e] = fmaf(treg[t], ui, oii[e]);
            oii[e] = fmaf(timg[t], ur, oii[e]);
          }
        float* col = outb + (int64_t)(kb + kk) * L2;
        if (vec) {
          *(float4*)(col + site0) = make_float4(orr[0], orr[1], orr[2], orr[3]);
          *(float4*)(col + L + site0) = make_float4(oii[0], oii[1], oii[2], oii[3]);
        } else {
          for (int e = 0; e < 4; ++e) {
            col[site0 + e] = orr[e];
            col[L + site0 + e] = oii[e];
          }
        }
        if (partial) {
#pragma unroll
          for (int e = 0; e < 4; ++e) accf[e] = fmaf(orr[e], orr[e], fmaf(oii[e], oii[e], accf[e]));
          if (++nacc == 16) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              acc2[e] += (double)accf[e];
              accf[e] = 0.f;
            }
            nacc = 0;
          }
        }
      }
    } else if (nval > 0)
      for (int kk = 0; kk < nk; ++kk) {
        const float* ar = sre[kk];
        const float* ai = sim[kk];
        float wr[4], wi[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {               // a short last group reads only its own run
          wr[e] = e < nval ? ar[base + e] : 0.f;
          wi[e] = e < nval ? ai[base + e] : 0.f;
        }
        float orr[4] = {0.f, 0.f, 0.f, 0.f}, oii[4] = {0.f, 0.f, 0.f, 0.f};
        for (int t = 0; t < ntap; ++t) {
          const float pr = tre[t], pi = tim[t];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            orr[e] = fmaf(pr, wr[e], orr[e]);
            orr[e] = fmaf(-pi, wi[e], orr[e]);
            oii[e] = fmaf(pr, wi[e], oii[e]);
            oii[e] = fmaf(pi, wr[e], oii[e]);
          }
          // slide the window one input down: inputs base - t - 1 .. base - t + 2
#pragma unroll
          for (int e = 3; e > 0; --e) {
            wr[e] = wr[e - 1];
            wi[e] = wi[e - 1];
          }
          if (t + 1 < ntap) {
            wr[0] = ar[base - t - 1];
            wi[0] = ai[base - t - 1];
          }
        }
        float* col = outb + (int64_t)(kb + kk) * L2;
        if (vec) {
          *(float4*)(col + site0) = make_float4(orr[0], orr[1], orr[2], orr[3]);
          *(float4*)(col + L + site0) = make_float4(oii[0], oii[1], oii[2], oii[3]);
        } else {
          for (int e = 0; e < nval; ++e) {
            col[site0 + e] = orr[e];
            col[L + site0 + e] = oii[e];
          }
        }
        if (partial) {
#pragma unroll
          for (int e = 0; e < 4; ++e) accf[e] = fmaf(orr[e], orr[e], fmaf(oii[e], oii[e], accf[e]));
          if (++nacc == 16) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              acc2[e] += (double)accf[e];
              accf[e] = 0.f;
            }
            nacc = 0;
          }
        }
      }
    if (more) {
      __syncthreads();                             // every thread is done with this stage
      store_stage(kb + kB4Cols);
      __syncthreads();
    }
  }
  if (partial)
    for (int e = 0; e < nval; ++e) partial[(b * nch + c) * L + site0 + e] = acc2[e] + (double)accf[e];
}

template <typename T, int LAYOUT, int SEGY>
__global__ void __launch_bounds__(256) band_y_kernel(const void* __restrict__ in, void* out, int L, int N, int Lx,
                                                     int Ly, const z64* __restrict__ taps,
                                                     const int* __restrict__ off, int ntap, int per,
                                                     double* partial, int nch, int tap_stride) {
  constexpr int H = SEGY + kBandMaxTaps - 1;
  __shared__ cplx<T> buf[H][32];
  __shared__ cplx<T> tp[kBandMaxTaps];
  const int64_t b = blockIdx.z;
  taps += b * tap_stride;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  if (tid < ntap) tp[tid] = cmk<T>((T)taps[tid].re, (T)taps[tid].im);
  const int nxt = (Lx + 31) / 32;
  const int xt = blockIdx.x % nxt, ys = blockIdx.x / nxt;
  const int x = xt * 32 + tx, y0 = ys * SEGY;
  const int offmax = off[0] + ntap - 1;
  const int h = SEGY + ntap - 1;
  const int c = blockIdx.y;
  const int k0 = c * per, k1 = min(N, k0 + per);
  // row sums of |out|^2 (see band_x4_kernel): in T over up to 16 columns, then double
  double s[SEGY / 8];
  T sf[SEGY / 8];
#pragma unroll
  for (int r = 0; r < SEGY / 8; ++r) {
    s[r] = 0.0;
    sf[r] = (T)0;
  }
  int nacc = 0;
  // staged rows of one column: h <= SEGY + kBandMaxTaps - 1, at most RY per thread, loaded
  // into registers before any is stored
  constexpr int RY = (H + 7) / 8;
  int srcr[RY];
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    int src = (y0 - offmax + ty + 8 * i) % Ly;
    srcr[i] = x + Lx * (src < 0 ? src + Ly : src);
  }
  for (int k = k0; k < k1; ++k) {
    cplx<T> v[RY];
#pragma unroll
    for (int i = 0; i < RY; ++i)
      if (x < Lx && ty + 8 * i < h) v[i] = band_io<T, LAYOUT>::ld(in, b, L, N, srcr[i], k);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RY; ++i)
      if (x < Lx && ty + 8 * i < h) buf[ty + 8 * i][tx] = v[i];
    __syncthreads();
    if (x < Lx)
#pragma unroll
      for (int r = 0; r < SEGY / 8; ++r) {
        const int yy = ty + 8 * r, y = y0 + yy;
        if (y < Ly) {
          cplx<T> acc = cmk<T>((T)0, (T)0);
          for (int t = 0; t < ntap; ++t) {
            const cplx<T> u = buf[yy + ntap - 1 - t][tx];
            acc.re += tp[t].re * u.re - tp[t].im * u.im;
            acc.im += tp[t].re * u.im + tp[t].im * u.re;
          }
          band_io<T, LAYOUT>::st(out, b, L, N, x + Lx * y, k, acc);
          if (partial) sf[r] += acc.re * acc.re + acc.im * acc.im;
        }
      }
    if (partial && ++nacc == 16) {
#pragma unroll
      for (int r = 0; r < SEGY / 8; ++r) {
        s[r] += (double)sf[r];
        sf[r] = (T)0;
      }
      nacc = 0;
    }
  }
  if (partial && x < Lx)
#pragma unroll
    for (int r = 0; r < SEGY / 8; ++r) {
      const int y = y0 + ty + 8 * r;
      if (y < Ly) partial[(b * nch + c) * L + x + Lx * y] = s[r] + (double)sf[r];
    }
}

namespace {
int clamp_chunks(int64_t blocks, int N) {
  const int64_t want = (8 * 152 + blocks - 1) / blocks;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, std::min(N, 128)));
}
}  // namespace

// the x stencil of the float state takes band_x4_kernel when its staged runs fit
bool use_band4(int Lx, int Ly, int layout, int ntap) {
  if (layout != 1) return false;
  const B4Shape g = band4_shape(Lx, Ly);
  const int runp = (g.S + ntap - 1 + 3) & ~3;
  return g.RB * runp + 4 <= kB4Pad;
}

int band_chunks(int Lx, int Ly, int N, int B, int dir, int layout) {
  int64_t blocks;
  if (dir == 0 && layout == 1) {
    const B4Shape g = band4_shape(Lx, Ly);
    blocks = (int64_t)g.segs * g.groups * B;
  } else {
    blocks = dir == 0 ? (int64_t)FM_CEIL_DIV(Lx, kBandSegX) * Ly * B
                      : (int64_t)FM_CEIL_DIV(Lx, 32) * FM_CEIL_DIV(Ly, seg_y(layout)) * B;
  }
  return clamp_chunks(blocks, N);
}

int site_chunks(int L, int N, int B) { return clamp_chunks((int64_t)FM_CEIL_DIV(L, 256) * B, N); }

cudaError_t band_propagate(cudaStream_t st, int layout, const void* in, void* out, int L, int N, int B, int Lx,
                           int Ly, int dir, const z64* taps, const int* off, int ntap, double* partial, int nch,
                           int tap_stride) {
  if (ntap < 1 || ntap > kBandMaxTaps || nch < 1 || Lx * Ly != L) return cudaErrorInvalidValue;
  const int per = FM_CEIL_DIV(N, nch);
  if (dir == 0 && use_band4(Lx, Ly, layout, ntap)) {
    const B4Shape g = band4_shape(Lx, Ly);
    const dim3 grid(g.segs * g.groups, nch, B);
    if (ntap == 15)                                // |J_r(0.1)| < 1e-15 from r = 8: the dt = 0.05 stencil
      band_x4_kernel<15><<<grid, 256, 0, st>>>((const float*)in, (float*)out, L, N, Lx, Ly, g.S, g.tpr, g.RB, g.segs,
                                               taps, off, ntap, per, partial, nch, tap_stride);
    else if (ntap == 17)
      band_x4_kernel<17><<<grid, 256, 0, st>>>((const float*)in, (float*)out, L, N, Lx, Ly, g.S, g.tpr, g.RB, g.segs,
                                               taps, off, ntap, per, partial, nch, tap_stride);
    else
      band_x4_kernel<0><<<grid, 256, 0, st>>>((const float*)in, (float*)out, L, N, Lx, Ly, g.S, g.tpr, g.RB, g.segs,
                                              taps, off, ntap, per, partial, nch, tap_stride);
  } else if (dir == 0) {
    const dim3 grid(FM_CEIL_DIV(Lx, kBandSegX) * Ly, nch, B);
    if (layout == 0)
      band_x_kernel<double, 0><<<grid, 256, 0, st>>>(in, out, L, N, Lx, taps, off, ntap, per, partial, nch,
                                                     tap_stride);
    else
      band_x_kernel<float, 1><<<grid, 256, 0, st>>>(in, out, L, N, Lx, taps, off, ntap, per, partial, nch,
                                                    tap_stride);
  } else {
    const dim3 grid(FM_CEIL_DIV(Lx, 32) * FM_CEIL_DIV(Ly, seg_y(layout)), nch, B);
    if (layout == 0)
      band_y_kernel<double, 0, seg_y(0)><<<grid, dim3(32, 8), 0, st>>>(in, out, L, N, Lx, Ly, taps, off, ntap, per,
                                                                       partial, nch, tap_stride);
    else
      band_y_kernel<float, 1, seg_y(1)><<<grid, dim3(32, 8), 0, st>>>(in, out, L, N, Lx, Ly, taps, off, ntap, per,
                                                                      partial, nch, tap_stride);
  }
  return cudaGetLastError();
}


// ------------------------------------------------------------------ Runge-Kutta step of Eq. (QSD_evo)
// One Horner stage of the fourth-order Taylor polynomial of X = A dt,
// A dt = -i dt H~ + diag(m), m_i = ln w_i (w = exp(m) from reduce_occupations):
//   out = U0 + c X Y,   (X Y)_i = -i dt J sum_{nearest neighbours j of i} Y_j + m_i Y_i.
// With c = 1/4, 1/3, 1/2, 1 in turn starting from Y = U0 the last stage gives
// U0 + X U0 + X^2 U0 / 2 + X^3 U0 / 6 + X^4 U0 / 24, the RK4 step of the linear
// constant-coefficient equation.  Neighbours x +- 1 (and y +- 1 on the torus),
// periodic; a direction of length 2 counts its one neighbour twice, as H~ does.
template <typename T, int LAYOUT>
__global__ void rk4_stage_kernel(const void* U0, const void* Y, void* out, int L, int N, int Lx, int Ly,
                                 const double* __restrict__ w, double dtJ, double c, int per) {
  const int64_t b = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L) return;
  const int x = i % Lx, y = i / Lx;
  const int xp = (x + 1) % Lx + Lx * y, xm = (x + Lx - 1) % Lx + Lx * y;
  const int yp = Ly > 1 ? x + Lx * ((y + 1) % Ly) : -1, ym = Ly > 1 ? x + Lx * ((y + Ly - 1) % Ly) : -1;
  const T m = (T)log(w[b * L + i]);
  const T h = (T)dtJ, cc = (T)c;
  const int k0 = blockIdx.y * per, k1 = min(N, k0 + per);
  for (int k = k0; k < k1; ++k) {
    cplx<T> s = cadd(band_io<T, LAYOUT>::ld(Y, b, L, N, xp, k), band_io<T, LAYOUT>::ld(Y, b, L, N, xm, k));
    if (yp >= 0) s = cadd(s, cadd(band_io<T, LAYOUT>::ld(Y, b, L, N, yp, k), band_io<T, LAYOUT>::ld(Y, b, L, N, ym, k)));
    const cplx<T> yi = band_io<T, LAYOUT>::ld(Y, b, L, N, i, k);
    // X Y = -i h s + m y_i
    const cplx<T> xy = cmk<T>(h * s.im + m * yi.re, -h * s.re + m * yi.im);
    const cplx<T> u0 = band_io<T, LAYOUT>::ld(U0, b, L, N, i, k);
    band_io<T, LAYOUT>::st(out, b, L, N, i, k, cmk<T>(u0.re + cc * xy.re, u0.im + cc * xy.im));
  }
}

cudaError_t rk4_stage(cudaStream_t st, int layout, const void* U0, const void* Y, void* out, int L, int N, int B,
                      int Lx, int Ly, const double* w, double dtJ, double c) {
  const int nch = site_chunks(L, N, B);
  const int per = FM_CEIL_DIV(N, nch);
  const dim3 grid(FM_CEIL_DIV(L, 256), nch, B);
  if (layout == 0)
    rk4_stage_kernel<double, 0><<<grid, 256, 0, st>>>(U0, Y, out, L, N, Lx, Ly, w, dtJ, c, per);
  else
    rk4_stage_kernel<float, 1><<<grid, 256, 0, st>>>(U0, Y, out, L, N, Lx, Ly, w, dtJ, c, per);
  return cudaGetLastError();
}

}  // namespace fm
