// Host-side launch wrappers of the device kernels (defined in
// pflbm_launch.cuh, instantiated for float and double in pflbm_f32.cu and
// pflbm_f64.cu).
#pragma once

#include <cuda_runtime.h>

#include "pflbm_kernels.cuh"

namespace pflbm {

template <typename T>
cudaError_t launch_march(int model, int mode, const Phys<T>& P, const Bufs<T>& B, cudaStream_t s);
// TMA-staged Allen-Cahn step (returns cudaErrorNotSupported when the grid is
// too narrow for it; the caller then uses launch_march)
template <typename T>
cudaError_t launch_step_tma(const Phys<T>& P, const Bufs<T>& B, int* err, bool unit_rates, cudaStream_t s);
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

}  // namespace pflbm
