// Definitions of the launch wrappers declared in pflbm_launch.h.
#pragma once

#include <cmath>

#include "pflbm_launch.h"

namespace pflbm {

template <class C, int MODEL>
static cudaError_t launch_march_model(int mode, const Phys<typename C::value_t>& P,
                                      const Bufs<typename C::value_t>& B, cudaStream_t s) {
  const dim3 grid((P.nx + BX - 1) / BX, (P.ny + LY - 1) / LY);
  switch (mode) {
    case MODE_STEP: k_march<C, MODEL, MODE_STEP><<<grid, BX, 0, s>>>(P, B); break;
    case MODE_MACRO: k_march<C, MODEL, MODE_MACRO><<<grid, BX, 0, s>>>(P, B); break;
    case MODE_HIST: k_march<C, MODEL, MODE_HIST><<<grid, BX, 0, s>>>(P, B); break;
    case MODE_INIT: k_march<C, MODEL, MODE_INIT><<<grid, BX, 0, s>>>(P, B); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_march(int model, int mode, const Phys<typename C::value_t>& P,
                         const Bufs<typename C::value_t>& B, cudaStream_t s) {
  return model == MODEL_CH ? launch_march_model<C, MODEL_CH>(mode, P, B, s)
                           : launch_march_model<C, MODEL_AC>(mode, P, B, s);
}

// Number of SMs of the current device (looked up once per device).
static inline int device_sm_count() {
  static int sms[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms[dev] = 152;
  return sms[dev];
}

// Rows per block segment: LY, halved (down to 8) until the grid of strips of
// `tbx` columns holds at least `waves` waves of `per_sm` resident blocks, so
// that grids of a few million nodes still fill every SM.  Each segment
// re-forms two phi rows and re-stages its first rows, so long segments are
// kept wherever the grid is large enough.
static inline int segment_rows(int nx, int ny, int tbx, int per_sm, int waves = 2) {
  const long long target = (long long)waves * device_sm_count() * per_sm;
  const long long strips = (nx + tbx - 1) / tbx;
  int seg = LY;
  while (seg > 8 && strips * ((ny + seg - 1) / seg) < target) seg /= 2;
  return seg;
}

// Rows per segment of the FP32 Allen-Cahn step on grids that hold fewer than
// eight waves of LY-row blocks: the length in [8, LY] with the least
// modelled time.  A block takes time in proportion to its rows plus two (the
// rows it re-stages first); blocks run in waves of (SMs x resident blocks),
// and a partial last wave of this latency-bound kernel costs about half a
// full wave beyond its share of the blocks.  Measured: 2048 x 1024 picks 23
// rows (26.2 GLUPS, 23.9 at 8), 4096 x 2048 picks 45 (28.1, 27.4 at 32).
static inline int segment_rows_waves(int nx, int ny, int tbx, int per_sm) {
  const long long slots = (long long)device_sm_count() * per_sm;
  const long long strips = (nx + tbx - 1) / tbx;
  if (strips * ((ny + LY - 1) / LY) >= 8 * slots) return LY;
  int pick = LY;
  double best = 0.0;
  for (int seg = LY; seg >= 8; --seg) {
    const double w = (double)(strips * ((ny + seg - 1) / seg)) / (double)slots;
    const double cost = (w + 0.5 * (std::ceil(w) - w)) * (seg + 2);
    if (seg == LY || cost < best) best = cost, pick = seg;  // ties keep the longer segment
  }
  return pick;
}

// Segment rows of the Allen-Cahn TMA step (with or without obstacles).  The
// 16-bit deviation step is bound by instruction issue, so blocks of a
// partial wave run faster and one wave of blocks suffices; FP64 keeps the
// two-wave rule.
template <class C>
static int tma_segment_rows(int nx, int ny) {
  using G = TmaCfg<C>;
  const int per_sm = G::threads / G::TBX;
  if (C::dev) return segment_rows(nx, ny, G::TBX, per_sm, 1);
  if (G::fp32) return segment_rows_waves(nx, ny, G::TBX, per_sm);
  return segment_rows(nx, ny, G::TBX, per_sm);
}

// Launch `kern` as a programmatic dependent of the kernel launched just
// before it on `s` (it may start once every block of that kernel has issued
// griddepcontrol.launch_dependents, and orders its reads of that kernel's
// output with griddepcontrol.wait), or as a plain launch.
template <typename... KArgs, typename... Args>
static cudaError_t launch_maybe_dependent(bool dependent, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                          cudaStream_t s, Args... args) {
  if (!dependent) {
    kern<<<grid, block, smem, s>>>(args...);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <class C, bool UR, bool VSEG, bool OBS = false>
static cudaError_t launch_tma_seg(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B,
                                  int* err, cudaStream_t s, bool dependent = false) {
  using G = TmaCfg<C>;
  using L = TmaLayout<C, G::TBX, G::DF, G::DG, G::slim>;
  // per function and device; cheap next to a step
  cudaError_t e = cudaFuncSetAttribute(k_step_tma<C, UR, VSEG, OBS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)L::bytes);
  if (e != cudaSuccess) return e;
  const dim3 grid((P.nx + G::TBX - 1) / G::TBX, (P.ny + P.seg_rows - 1) / P.seg_rows);
  // a programmatic dependent of the kernel before it: without obstacles the
  // previous step (its blocks start during that step's last blocks and wait
  // for it to finish), with obstacles the phi pass (the blocks away from the
  // obstacle start while the pass finishes; the near blocks wait for it
  // before reading its plane)
  return launch_maybe_dependent(!OBS || dependent, k_step_tma<C, UR, VSEG, OBS>, grid, dim3(G::TBX), L::bytes, s, P,
                                B, err);
}

// Segments of LY rows use the instantiation with the constant length (its
// register allocation is the tuned one); shorter ones the runtime-length one.
template <class C, bool UR, bool OBS = false>
static cudaError_t launch_tma_variant(const Phys<typename C::value_t>& P0, const Bufs<typename C::value_t>& B,
                                      int* err, cudaStream_t s, bool dependent = false) {
  Phys<typename C::value_t> P = P0;
  P.seg_rows = tma_segment_rows<C>(P.nx, P.ny);
  return P.seg_rows == LY ? launch_tma_seg<C, UR, false, OBS>(P, B, err, s, dependent)
                          : launch_tma_seg<C, UR, true, OBS>(P, B, err, s, dependent);
}

// Launch grid of the Allen-Cahn TMA step (strip width, rows per segment).
template <class C>
void tma_step_grid(int nx, int ny, int* tbx, int* seg_rows) {
  *tbx = TmaCfg<C>::TBX;
  *seg_rows = tma_segment_rows<C>(nx, ny);
}

// Launch grid of the Cahn-Hilliard TMA step.
template <class C>
static int tma_ch_segment_rows(int nx, int ny);
template <class C>
void tma_ch_step_grid(int nx, int ny, int* tbx, int* seg_rows) {
  *tbx = TmaChCfg<C>::TBX;
  *seg_rows = tma_ch_segment_rows<C>(nx, ny);
}

// Cahn-Hilliard step: same segment rule, its own launch shape (TmaChCfg).
template <class C>
static int tma_ch_segment_rows(int nx, int ny) {
  using G = TmaChCfg<C>;
  return segment_rows(nx, ny, G::TBX, G::threads / G::TBX);
}

template <class C, bool UR, bool VSEG, bool OBS = false>
static cudaError_t launch_tma_ch_seg(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B,
                                     int* err, cudaStream_t s, bool dependent = false) {
  using G = TmaChCfg<C>;
  using L = TmaChLayout<C, G::TBX, G::DF, G::DG>;
  cudaError_t e = cudaFuncSetAttribute(k_step_tma_ch<C, UR, VSEG, OBS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  const dim3 grid((P.nx + G::TBX - 1) / G::TBX, (P.ny + P.seg_rows - 1) / P.seg_rows);
  return launch_maybe_dependent(!OBS || dependent, k_step_tma_ch<C, UR, VSEG, OBS>, grid, dim3(G::TBX), L::bytes, s,
                                P, B, err);
}

template <class C>
cudaError_t launch_step_tma_ch(const Phys<typename C::value_t>& P0, const Bufs<typename C::value_t>& B, int* err,
                               bool unit_rates, cudaStream_t s) {
  if (P0.nx < 4 * XPAD) return cudaErrorNotSupported;
  Phys<typename C::value_t> P = P0;
  P.seg_rows = tma_ch_segment_rows<C>(P.nx, P.ny);
  if (P.seg_rows == LY)
    return unit_rates ? launch_tma_ch_seg<C, true, false>(P, B, err, s) : launch_tma_ch_seg<C, false, false>(P, B, err, s);
  return unit_rates ? launch_tma_ch_seg<C, true, true>(P, B, err, s) : launch_tma_ch_seg<C, false, true>(P, B, err, s);
}

// The launch shape per storage codec (strip width, staging depth, blocks
// per SM) and the measurements behind it are given with TmaCfg.
template <class C>
cudaError_t launch_step_tma(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B, int* err,
                            bool unit_rates, cudaStream_t s) {
  if (P.nx < 4 * XPAD) return cudaErrorNotSupported;
  return unit_rates ? launch_tma_variant<C, true>(P, B, err, s) : launch_tma_variant<C, false>(P, B, err, s);
}

static inline dim3 row_grid(int nx, int ny, int threads) { return dim3((nx + threads - 1) / threads, ny); }

template <class C>
cudaError_t launch_pull_export(const Phys<typename C::value_t>& P, const void* in, int set, int k, double* out,
                               double add, int x0, int y0, int w, int hgt, cudaStream_t s) {
  k_pull_export<C><<<row_grid(w, hgt, 128), 128, 0, s>>>(P, in, set, k, out, add, x0, y0, w, hgt);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_restream(const Phys<typename C::value_t>& P, const typename C::value_t* in, void* out,
                            int set, cudaStream_t s) {
  k_restream<C><<<row_grid(P.nx, P.ny, 128), 128, 0, s>>>(P, in, out, set);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pull(const Phys<T>& P, const T* in, T* out, cudaStream_t s) {
  k_pull<T><<<row_grid(P.nx, P.ny, 128), 128, 0, s>>>(P, in, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_unstream(const Phys<T>& P, const T* in, T* out, cudaStream_t s) {
  k_unstream<T><<<row_grid(P.nx, P.ny, 128), 128, 0, s>>>(P, in, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_export(const Phys<T>& P, const T* in, int NP, int k, double* out, double add,
                          int x0, int y0, int w, int hgt, cudaStream_t s) {
  k_export<T><<<row_grid(w, hgt, 128), 128, 0, s>>>(P, in, NP, k, out, add, x0, y0, w, hgt);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_import(const Phys<T>& P, const double* in, T* out, int NP, int k, double sub,
                          cudaStream_t s) {
  k_import<T><<<row_grid(P.nx, P.ny, 128), 128, 0, s>>>(P, in, out, NP, k, sub);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag(const Phys<T>& P, const T* macro, const T* phi_prev, double* partial,
                        int nparts, double* out, cudaStream_t s) {
  k_diag_partial<T><<<nparts, DIAG_THREADS, 0, s>>>(P, macro, phi_prev, partial);
  k_diag_final<T><<<1, DIAG_THREADS, 0, s>>>(partial, nparts, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_obs_links(const Phys<T>& P, const unsigned char* solid, uint16_t* obs, cudaStream_t s) {
  k_obs_links<T><<<row_grid(P.nx, P.ny, OBS_THREADS), OBS_THREADS, 0, s>>>(P, solid, obs);
  return cudaGetLastError();
}

template <class C, int MODEL, int MODE, bool UR>
static cudaError_t obs_passes(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B,
                              typename C::value_t* phis, typename C::value_t* mus, cudaStream_t s) {
  using T = typename C::value_t;
  const dim3 grid = row_grid(P.nx, P.ny, OBS_THREADS);
  const int fill_blocks = (P.obs_nfill + OBS_THREADS - 1) / OBS_THREADS;
  k_obs_phi<C, MODE == MODE_INIT ? MODE_INIT : MODE_STEP><<<grid, OBS_THREADS, 0, s>>>(P, B, phis, 0, P.nx, 0);
  if (MODEL == MODEL_CH) {
    k_obs_mu<T><<<grid, OBS_THREADS, 0, s>>>(P, phis, mus, 0, P.nx, 0);
    if (fill_blocks) k_obs_fill<T><<<fill_blocks, OBS_THREADS, 0, s>>>(P, mus);
  }
  k_obs_node<C, MODEL, MODE, UR><<<grid, OBS_THREADS, 0, s>>>(P, B, phis, mus);
  return cudaGetLastError();
}

template <class C, int MODEL>
static cudaError_t obs_model(int mode, const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B,
                             typename C::value_t* phis, typename C::value_t* mus, bool unit_rates,
                             cudaStream_t s) {
  switch (mode) {
    case MODE_STEP:
      return unit_rates ? obs_passes<C, MODEL, MODE_STEP, true>(P, B, phis, mus, s)
                        : obs_passes<C, MODEL, MODE_STEP, false>(P, B, phis, mus, s);
    case MODE_MACRO: return obs_passes<C, MODEL, MODE_MACRO, false>(P, B, phis, mus, s);
    case MODE_HIST: return obs_passes<C, MODEL, MODE_HIST, false>(P, B, phis, mus, s);
    case MODE_INIT: return obs_passes<C, MODEL, MODE_INIT, false>(P, B, phis, mus, s);
    default: return cudaErrorInvalidValue;
  }
}

// Allen-Cahn step with obstacles on the TMA kernel: phi and its fill over
// the region the blocks near obstacles read (P.obs_box; the whole grid
// without P.obs_near), then k_step_tma<..., OBS>, whose near blocks read phi
// from the plane and the others run the plain step's path.
template <class C>
static cudaError_t obs_step_tma(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B0,
                                typename C::value_t* phis, int* err, bool unit_rates, cudaStream_t s) {
  using T = typename C::value_t;
  const int x_lo = P.obs_near ? P.obs_box[0] : 0, x_hi = P.obs_near ? P.obs_box[1] : P.nx;
  const int y_lo = P.obs_near ? P.obs_box[2] : 0, y_hi = P.obs_near ? P.obs_box[3] : P.ny;
  const bool pass = x_hi > x_lo && y_hi > y_lo;
  if (pass)
    k_obs_phi<C, MODE_STEP><<<row_grid(x_hi - x_lo, y_hi - y_lo, OBS_THREADS), OBS_THREADS, 0, s>>>(P, B0, phis, x_lo,
                                                                                                   x_hi, y_lo);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  Bufs<T> B = B0;
  B.phis = phis;
  // the step is the phi pass's programmatic dependent only right after it
  return unit_rates ? launch_tma_variant<C, true, true>(P, B, err, s, pass)
                    : launch_tma_variant<C, false, true>(P, B, err, s, pass);
}

// Cahn-Hilliard step with obstacles on the TMA kernel: phi with its fill and
// mu_phi over the regions the blocks near obstacles read (P.obs_box,
// P.obs_box_mu; the whole grid without P.obs_near), the mu_phi fill, then
// k_step_tma_ch<..., OBS>, whose near blocks read both planes and the
// others run the plain step's path.
template <class C>
static cudaError_t obs_step_tma_ch(const Phys<typename C::value_t>& P0, const Bufs<typename C::value_t>& B0,
                                   typename C::value_t* phis, typename C::value_t* mus, int* err, bool unit_rates,
                                   cudaStream_t s) {
  using T = typename C::value_t;
  const bool nb = P0.obs_near != nullptr;
  const int* bp = P0.obs_box;
  const int* bm = P0.obs_box_mu;
  const int px0 = nb ? bp[0] : 0, px1 = nb ? bp[1] : P0.nx, py0 = nb ? bp[2] : 0, py1 = nb ? bp[3] : P0.ny;
  const int mx0 = nb ? bm[0] : 0, mx1 = nb ? bm[1] : P0.nx, my0 = nb ? bm[2] : 0, my1 = nb ? bm[3] : P0.ny;
  const int fill_blocks = (P0.obs_nfill + OBS_THREADS - 1) / OBS_THREADS;
  // phi pass (a plain launch: it reads the previous step's populations),
  // then the mu_phi pass, the fill and the step, each a programmatic
  // dependent of the kernel before it (each waits for that kernel's output)
  bool prev = false;  // a pass was launched just before
  cudaError_t e = cudaSuccess;
  if (px1 > px0 && py1 > py0) {
    k_obs_phi<C, MODE_STEP><<<row_grid(px1 - px0, py1 - py0, OBS_THREADS), OBS_THREADS, 0, s>>>(P0, B0, phis, px0,
                                                                                               px1, py0);
    e = cudaGetLastError();
    prev = true;
  }
  if (e == cudaSuccess && mx1 > mx0 && my1 > my0) {
    e = launch_maybe_dependent(prev, k_obs_mu<T>, row_grid(mx1 - mx0, my1 - my0, OBS_THREADS), dim3(OBS_THREADS), 0, s,
                               P0, (const T*)phis, mus, mx0, mx1, my0);
    prev = true;
  }
  if (e == cudaSuccess && fill_blocks) {
    e = launch_maybe_dependent(prev, k_obs_fill<T>, dim3(fill_blocks), dim3(OBS_THREADS), 0, s, P0, mus);
    prev = true;
  }
  if (e != cudaSuccess) return e;
  Bufs<T> B = B0;
  B.phis = phis;
  B.mus = mus;
  Phys<T> P = P0;
  P.seg_rows = tma_ch_segment_rows<C>(P.nx, P.ny);
  if (P.seg_rows == LY)
    return unit_rates ? launch_tma_ch_seg<C, true, false, true>(P, B, err, s, prev)
                      : launch_tma_ch_seg<C, false, false, true>(P, B, err, s, prev);
  return unit_rates ? launch_tma_ch_seg<C, true, true, true>(P, B, err, s, prev)
                    : launch_tma_ch_seg<C, false, true, true>(P, B, err, s, prev);
}

template <class C>
cudaError_t launch_obs(int model, int mode, const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B,
                       typename C::value_t* phis, typename C::value_t* mus, bool unit_rates, int* err,
                       bool use_tma, cudaStream_t s) {
  if (!P.obs || !phis || (model == MODEL_CH && !mus)) return cudaErrorInvalidValue;
  if (use_tma && model == MODEL_AC && mode == MODE_STEP && P.nx >= 4 * XPAD)
    return obs_step_tma<C>(P, B, phis, err, unit_rates, s);
  if (use_tma && model == MODEL_CH && mode == MODE_STEP && P.nx >= 4 * XPAD)
    return obs_step_tma_ch<C>(P, B, phis, mus, err, unit_rates, s);
  return model == MODEL_CH ? obs_model<C, MODEL_CH>(mode, P, B, phis, mus, unit_rates, s)
                           : obs_model<C, MODEL_AC>(mode, P, B, phis, mus, unit_rates, s);
}

// One adjoint step (or, with hist_only, the adjoint of the history set-up at
// t = 0 without the reverse streaming).  state: snapshot of the step's input
// state (f* set, g* set of pop_bytes each, then the 5 history planes).
template <typename T>
cudaError_t launch_adjoint_step(const Phys<T>& P, const void* state, long long pop_bytes, const AdjBufs& A,
                                double* gacc, bool hist_only, cudaStream_t s) {
  const T* fin = static_cast<const T*>(state);
  const T* gin = reinterpret_cast<const T*>(static_cast<const unsigned char*>(state) + pop_bytes);
  const T* hist = reinterpret_cast<const T*>(static_cast<const unsigned char*>(state) + 2 * pop_bytes);
  T* phi = static_cast<T*>(A.phi);
  T* lext = static_cast<T*>(A.lext);
  const dim3 grid((P.nx + ADJ_THREADS - 1) / ADJ_THREADS, P.ny);
  k_adj_phi<T><<<grid, ADJ_THREADS, 0, s>>>(P, fin, phi);
  k_adj_node<T><<<grid, ADJ_THREADS, 0, s>>>(P, fin, gin, hist, phi, static_cast<const T*>(A.lf),
                                             static_cast<const T*>(A.lg), static_cast<T*>(A.lh),
                                             static_cast<T*>(A.lp9), static_cast<T*>(A.lfp),
                                             static_cast<T*>(A.lgp), A.gpart, hist_only ? 1 : 0);
  const int ex = P.nx + 2 * P.wall_x, ey = P.ny + 2 * P.wall_y;
  k_adj_gather<T><<<dim3((ex + ADJ_THREADS - 1) / ADJ_THREADS, ey), ADJ_THREADS, 0, s>>>(
      P, static_cast<const T*>(A.lp9), lext);
  if (P.wall_y) k_adj_fold_y<T><<<(ex + ADJ_THREADS - 1) / ADJ_THREADS, ADJ_THREADS, 0, s>>>(P, phi, lext);
  if (P.wall_x) k_adj_fold_x<T><<<(P.ny + ADJ_THREADS - 1) / ADJ_THREADS, ADJ_THREADS, 0, s>>>(P, phi, lext);
  if (!hist_only)
    k_adj_stream<T><<<grid, ADJ_THREADS, 0, s>>>(P, static_cast<const T*>(A.lfp), static_cast<const T*>(A.lgp),
                                                 lext, static_cast<T*>(A.lf), static_cast<T*>(A.lg));
  k_adj_reduce<T><<<1, 256, 0, s>>>(A.gpart, (long long)grid.x * grid.y, gacc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_seed(const Phys<T>& P, const double* djdphi, const AdjBufs& A, cudaStream_t s) {
  const dim3 grid((P.nx + ADJ_THREADS - 1) / ADJ_THREADS, P.ny);
  k_adj_seed<T><<<grid, ADJ_THREADS, 0, s>>>(P, djdphi, static_cast<T*>(A.lf), static_cast<T*>(A.lg),
                                             static_cast<T*>(A.lh));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adjoint_init(const Phys<T>& P, const AdjBufs& A, double* out, cudaStream_t s) {
  const dim3 grid((P.nx + ADJ_THREADS - 1) / ADJ_THREADS, P.ny);
  k_adj_init<T><<<grid, ADJ_THREADS, 0, s>>>(P, static_cast<const T*>(A.lf), static_cast<const T*>(A.lext), out);
  return cudaGetLastError();
}

// the codec-typed wrappers of one storage codec
#define PFLBM_INSTANTIATE_CODEC(C)                                                                  \
  template cudaError_t launch_march<C>(int, int, const Phys<C::value_t>&, const Bufs<C::value_t>&,  \
                                       cudaStream_t);                                               \
  template cudaError_t launch_step_tma<C>(const Phys<C::value_t>&, const Bufs<C::value_t>&, int*,   \
                                          bool, cudaStream_t);                                      \
  template cudaError_t launch_step_tma_ch<C>(const Phys<C::value_t>&, const Bufs<C::value_t>&, int*, \
                                             bool, cudaStream_t);                                   \
  template cudaError_t launch_obs<C>(int, int, const Phys<C::value_t>&, const Bufs<C::value_t>&,    \
                                     C::value_t*, C::value_t*, bool, int*, bool, cudaStream_t);     \
  template void tma_step_grid<C>(int, int, int*, int*);                                               \
  template void tma_ch_step_grid<C>(int, int, int*, int*);

#define PFLBM_INSTANTIATE_DEV(C)                                                                    \
  PFLBM_INSTANTIATE_CODEC(C)                                                                        \
  template cudaError_t launch_pull_export<C>(const Phys<C::value_t>&, const void*, int, int, double*, \
                                             double, int, int, int, int, cudaStream_t);             \
  template cudaError_t launch_restream<C>(const Phys<C::value_t>&, const C::value_t*, void*, int,   \
                                          cudaStream_t);

// the arithmetic-type wrappers
#define PFLBM_INSTANTIATE(T)                                                                        \
  PFLBM_INSTANTIATE_CODEC(PopPlain<T>)                                                              \
  template cudaError_t launch_pull<T>(const Phys<T>&, const T*, T*, cudaStream_t);                \
  template cudaError_t launch_unstream<T>(const Phys<T>&, const T*, T*, cudaStream_t);            \
  template cudaError_t launch_export<T>(const Phys<T>&, const T*, int, int, double*, double, int,  \
                                        int, int, int, cudaStream_t);                              \
  template cudaError_t launch_import<T>(const Phys<T>&, const double*, T*, int, int, double,      \
                                        cudaStream_t);                                             \
  template cudaError_t launch_diag<T>(const Phys<T>&, const T*, const T*, double*, int, double*,  \
                                      cudaStream_t);                                             \
  template cudaError_t launch_adjoint_step<T>(const Phys<T>&, const void*, long long, const AdjBufs&, \
                                              double*, bool, cudaStream_t);                       \
  template cudaError_t launch_adjoint_seed<T>(const Phys<T>&, const double*, const AdjBufs&,      \
                                              cudaStream_t);                                      \
  template cudaError_t launch_adjoint_init<T>(const Phys<T>&, const AdjBufs&, double*, cudaStream_t); \
  template cudaError_t launch_obs_links<T>(const Phys<T>&, const unsigned char*, uint16_t*, cudaStream_t);

}  // namespace pflbm
