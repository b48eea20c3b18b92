// Host-side launch wrappers of the device kernels (defined in
// pflbm_launch.cuh).  C is a population storage codec (PopPlain<float>,
// PopPlain<double>, PopDev<__half>, PopDev<__nv_bfloat16>); each is
// instantiated in a translation unit of its own (pflbm_f32.cu, pflbm_f64.cu,
// pflbm_f16.cu, pflbm_bf16.cu).  T-typed wrappers handle the planes kept in
// the arithmetic type (history, macroscopic fields, diagnostics).
#pragma once

#include <cuda_runtime.h>

#include "pflbm_kernels.cuh"
#include "pflbm_adjoint.cuh"
#include "pflbm_obstacle.cuh"

namespace pflbm {

template <class C>
cudaError_t launch_march(int model, int mode, const Phys<typename C::value_t>& P,
                         const Bufs<typename C::value_t>& B, cudaStream_t s);
// TMA-staged Allen-Cahn step (returns cudaErrorNotSupported when the grid is
// too narrow for it; the caller then uses launch_march)
template <class C>
cudaError_t launch_step_tma(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B, int* err,
                            bool unit_rates, cudaStream_t s);
// its launch grid: strip width and rows per segment on the current device
template <class C>
void tma_step_grid(int nx, int ny, int* tbx, int* seg_rows);
// the Cahn-Hilliard step's launch grid
template <class C>
void tma_ch_step_grid(int nx, int ny, int* tbx, int* seg_rows);
// TMA-staged Cahn-Hilliard step (the same contract)
template <class C>
cudaError_t launch_step_tma_ch(const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B, int* err,
                               bool unit_rates, cudaStream_t s);
// deviation storage: pulled plane k of a set -> dense doubles of a region
template <class C>
cudaError_t launch_pull_export(const Phys<typename C::value_t>& P, const void* in, int set, int k, double* out,
                               double add, int x0, int y0, int w, int hgt, cudaStream_t s);
// deviation storage: pulled values (9 plain planes) -> encoded post-collision set
template <class C>
cudaError_t launch_restream(const Phys<typename C::value_t>& P, const typename C::value_t* in, void* out,
                            int set, cudaStream_t s);
template <typename T>
cudaError_t launch_pull(const Phys<T>& P, const T* in, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_unstream(const Phys<T>& P, const T* in, T* out, cudaStream_t s);
// plane k of a set of NP row-interleaved planes <-> dense doubles
template <typename T>
cudaError_t launch_export(const Phys<T>& P, const T* in, int NP, int k, double* out, double add,
                          int x0, int y0, int w, int hgt, cudaStream_t s);
template <typename T>
cudaError_t launch_import(const Phys<T>& P, const double* in, T* out, int NP, int k, double sub,
                          cudaStream_t s);
template <typename T>
cudaError_t launch_diag(const Phys<T>& P, const T* macro, const T* phi_prev, double* partial,
                        int nparts, double* out, cudaStream_t s);
// solid obstacles (pflbm_obstacle.cuh): the reflecting links of every node
// from a dense byte mask, and one step (or MACRO / HIST / INIT pass) through
// the obstacle passes; phis, mus: one-plane work planes of the arithmetic
// type.  With use_tma the Allen-Cahn step runs its node update on the TMA
// kernel (err: its time-out flag).
template <typename T>
cudaError_t launch_obs_links(const Phys<T>& P, const unsigned char* solid, uint16_t* obs, cudaStream_t s);
template <class C>
cudaError_t launch_obs(int model, int mode, const Phys<typename C::value_t>& P, const Bufs<typename C::value_t>& B,
                       typename C::value_t* phis, typename C::value_t* mus, bool unit_rates, int* err,
                       bool use_tma, cudaStream_t s);
// discrete adjoint of the Allen-Cahn step (pflbm_adjoint.cuh), plain storage
template <typename T>
cudaError_t launch_adjoint_step(const Phys<T>& P, const void* state, long long pop_bytes, const AdjBufs& A,
                                double* gacc, bool hist_only, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint_seed(const Phys<T>& P, const double* djdphi, const AdjBufs& A, cudaStream_t s);
template <typename T>
cudaError_t launch_adjoint_init(const Phys<T>& P, const AdjBufs& A, double* out, cudaStream_t s);

}  // namespace pflbm
