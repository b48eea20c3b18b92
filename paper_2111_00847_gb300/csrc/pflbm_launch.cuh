// Definitions of the launch wrappers declared in pflbm_launch.h.
#pragma once

#include "pflbm_launch.h"

namespace pflbm {

template <typename T, int MODEL>
static cudaError_t launch_march_model(int mode, const Phys<T>& P, const Bufs<T>& B, cudaStream_t s) {
  const dim3 grid((P.nx + BX - 1) / BX, (P.ny + LY - 1) / LY);
  switch (mode) {
    case MODE_STEP: k_march<T, MODEL, MODE_STEP><<<grid, BX, 0, s>>>(P, B); break;
    case MODE_MACRO: k_march<T, MODEL, MODE_MACRO><<<grid, BX, 0, s>>>(P, B); break;
    case MODE_HIST: k_march<T, MODEL, MODE_HIST><<<grid, BX, 0, s>>>(P, B); break;
    case MODE_INIT: k_march<T, MODEL, MODE_INIT><<<grid, BX, 0, s>>>(P, B); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_march(int model, int mode, const Phys<T>& P, const Bufs<T>& B, cudaStream_t s) {
  return model == MODEL_CH ? launch_march_model<T, MODEL_CH>(mode, P, B, s)
                           : launch_march_model<T, MODEL_AC>(mode, P, B, s);
}

template <typename T, bool UR, int TBX, int DF, int DG>
static cudaError_t launch_tma_variant(const Phys<T>& P, const Bufs<T>& B, int* err, cudaStream_t s) {
  using L = TmaLayout<T, TBX, DF, DG>;
  // per function and device; cheap next to a step
  cudaError_t e = cudaFuncSetAttribute(k_step_tma<T, UR, TBX, DF, DG>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  const dim3 grid((P.nx + TBX - 1) / TBX, (P.ny + LY - 1) / LY);
  k_step_tma<T, UR, TBX, DF, DG><<<grid, TBX, L::bytes, s>>>(P, B, err);
  return cudaGetLastError();
}

// Strip of 160 columns (5 warps), f and g rows staged one march step ahead:
// 56 KB of shared memory per FP32 block, four blocks (20 warps) per SM.
// Measured on the 16384^2 FP32 step against the alternatives (GLUPS):
// 160/1/1 29.5; 128 columns with f two steps ahead (4 blocks) 28.0, with
// both one ahead (5 blocks) 27.2; 96 columns (6 blocks) 28.2; 192 (3 blocks)
// 27.6; 256 (2 blocks) 27.5; 160 with f two ahead (3 blocks) 24.9.
constexpr int TMA_TBX = 160, TMA_DF = 1, TMA_DG = 1;

template <typename T>
cudaError_t launch_step_tma(const Phys<T>& P, const Bufs<T>& B, int* err, bool unit_rates, cudaStream_t s) {
  if (P.nx < 4 * XPAD) return cudaErrorNotSupported;
  return unit_rates ? launch_tma_variant<T, true, TMA_TBX, TMA_DF, TMA_DG>(P, B, err, s)
                    : launch_tma_variant<T, false, TMA_TBX, TMA_DF, TMA_DG>(P, B, err, s);
}

static inline dim3 row_grid(int nx, int ny, int threads) { return dim3((nx + threads - 1) / threads, ny); }

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

#define PFLBM_INSTANTIATE(T)                                                                        \
  template cudaError_t launch_march<T>(int, int, const Phys<T>&, const Bufs<T>&, cudaStream_t);   \
  template cudaError_t launch_step_tma<T>(const Phys<T>&, const Bufs<T>&, int*, bool, cudaStream_t);  \
  template cudaError_t launch_pull<T>(const Phys<T>&, const T*, T*, cudaStream_t);                \
  template cudaError_t launch_unstream<T>(const Phys<T>&, const T*, T*, cudaStream_t);            \
  template cudaError_t launch_export<T>(const Phys<T>&, const T*, int, int, double*, double, int,  \
                                        int, int, int, cudaStream_t);                              \
  template cudaError_t launch_import<T>(const Phys<T>&, const double*, T*, int, int, double,      \
                                        cudaStream_t);                                             \
  template cudaError_t launch_diag<T>(const Phys<T>&, const T*, const T*, double*, int, double*,  \
                                      cudaStream_t);

}  // namespace pflbm
