// Solid obstacles: the step on a grid where some nodes are solid.
//
// A solid node takes no part in the flow.  A link whose upstream node is
// solid reflects like a wall link (half-way bounce-back, Sec. 4); the
// reflecting links of every node are precomputed once per mask (P.obs, see
// Phys).  The paper states the wetting condition for plane walls only (Eqs.
// (49)-(50)); at a solid node the stencils of Eqs. (C.9)-(C.10) see the
// neutral-wetting value of the field: the mean over the fluid nodes among
// its four axis neighbours, or, with none, over its fluid diagonal
// neighbours.  Next to a plane of solid nodes this is the mirror value, the
// theta = 90 degrees ghost of Eq. (50).  Every per-node output of a solid
// node is zero.
//
// The fill needs phi (and, for Cahn-Hilliard, mu_phi) of fluid nodes two
// (three) nodes away, so these fields are first formed on planes, one thread
// per node:
//   k_obs_phi   phi = sum_i f_i at fluid nodes (Eq. (22a)) and its
//               neutral-wetting value at the solid nodes next to fluid
//               -> phi plane
//   k_obs_mu    (CH) mu_phi of Eq. (5) at fluid nodes -> mu plane, then
//   k_obs_fill  its neutral-wetting values
// The step's node update then runs on the TMA step kernels instantiated with
// OBS (pflbm_kernels.cuh).  There only the blocks near an obstacle read the
// planes (the others run the plain step's path), so per step the passes
// cover only the regions those blocks read.  k_obs_node is the same update
// one thread per node: the initial state, history and macroscopic passes,
// and the step under LBM_FLAG_NO_TMA or on grids under 16 columns, with the
// passes over whole planes.  It takes the stencils from the planes with the
// wall ghosts of Eq. (50) (mirror for mu_phi), pulls with reflection at
// solid links, collides and stores.
#pragma once

#include "pflbm_kernels.cuh"

namespace pflbm {

constexpr int OBS_THREADS = 128;

// Reflecting links and the solid bit of every node from a dense byte mask.
template <typename T>
__global__ void k_obs_links(const Phys<T> P, const unsigned char* __restrict__ solid, uint16_t* __restrict__ obs) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  unsigned m = solid[(long long)y * P.nx + x] ? (1u << OBS_SOLID) : 0u;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    int sx = x - cx[i], sy = y - cy[i];
    bool refl = false;
    if (sx < 0 || sx >= P.nx) {
      if (P.wall_x) refl = true;
      else sx = sx < 0 ? sx + P.nx : sx - P.nx;
    }
    if (sy < 0 || sy >= P.ny) {
      if (P.wall_y) refl = true;
      else sy = sy < 0 ? sy + P.ny : sy - P.ny;
    }
    if (!refl && solid[(long long)sy * P.nx + sx]) refl = true;
    if (refl) m |= 1u << (i - 1);
  }
  obs[(long long)y * P.nx + x] = (uint16_t)m;
}

// phi at every fluid node of [x_lo, x_hi) x [y_lo, y_hi) (INIT: the given
// field), and at every solid node there with a fluid neighbour the
// neutral-wetting value of reading 17: the mean over its fluid axis
// neighbours, or, with none, over its fluid diagonal neighbours.  A solid
// node forms its neighbours' phi again from their own pulls (the same sum9,
// so the same bits as the neighbours store), so phi and its fill take one
// pass.  Neighbour x + c_k is fluid when link opp(k) of the node does not
// reflect.  The plane has the one-plane row layout ix(P, 1, 0, x, y).
template <class C, int MODE>
__device__ __forceinline__ typename C::value_t obs_phi_node(const Phys<typename C::value_t>& P,
                                                            const Bufs<typename C::value_t>& B, int x, int y,
                                                            unsigned m) {
  using T = typename C::value_t;
  if (MODE == MODE_INIT) return T(B.iphi[(long long)y * P.nx + x]);
  T f[9];
  pull9_obs<C>(B.fin, P, 0, x, y, m, f);
  return sum9(f);
}

// Over the nodes [x_lo, x_hi) x [y_lo, y_hi) of the grid (blockIdx.y: the row).
template <class C, int MODE>
__global__ void k_obs_phi(const Phys<typename C::value_t> P, const Bufs<typename C::value_t> B,
                          typename C::value_t* __restrict__ phis, int x_lo, int x_hi, int y_lo) {
  using T = typename C::value_t;
  // a step kernel launched as this pass's programmatic dependent may start
  // now; it waits for this grid before it reads the plane
  asm volatile("griddepcontrol.launch_dependents;");
  const int x = x_lo + blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y_lo + blockIdx.y;
  if (x >= x_hi) return;
  const unsigned m = P.obs[(long long)y * P.nx + x];
  if (!((m >> OBS_SOLID) & 1u)) {
    phis[ix(P, 1, 0, x, y)] = obs_phi_node<C, MODE>(P, B, x, y, m);
    return;
  }
  if ((m & 0xffu) == 0xffu) return;  // no fluid neighbour: no fluid stencil reads this node
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  T val = T(0);
  for (int k0 = 1; k0 <= 5; k0 += 4) {
    T sm = T(0);
    int c = 0;
    for (int k = k0; k < k0 + 4; ++k) {
      if ((m >> (op[k] - 1)) & 1u) continue;
      int xn = x + cx[k], yn = y + cy[k];
      xn = xn < 0 ? xn + P.nx : (xn >= P.nx ? xn - P.nx : xn);
      yn = yn < 0 ? yn + P.ny : (yn >= P.ny ? yn - P.ny : yn);
      sm += obs_phi_node<C, MODE>(P, B, xn, yn, P.obs[(long long)yn * P.nx + xn]);
      ++c;
    }
    if (c > 0) {
      val = sm / T(c);
      break;
    }
  }
  phis[ix(P, 1, 0, x, y)] = val;
}

// Neutral-wetting value at each solid node next to fluid (P.obs_fill), from
// the fluid nodes of the same plane (reads fluid entries only, writes solid
// entries only).  Neighbour x + c_k is fluid when link opp(k) of the node
// does not reflect.
template <typename T>
__global__ void k_obs_fill(const Phys<T> P, T* __restrict__ pl) {
  // launched as the programmatic dependent of the pass before it (and as the
  // primary of the step after it): let the next kernel start, wait for the
  // previous one's plane
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.obs_nfill) return;
  const int n = P.obs_fill[t];
  const int y = n / P.nx, x = n - y * P.nx;
  const unsigned m = P.obs[n];
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  T val = T(0);
  for (int k0 = 1; k0 <= 5; k0 += 4) {
    T s = T(0);
    int c = 0;
    for (int k = k0; k < k0 + 4; ++k) {
      if ((m >> (op[k] - 1)) & 1u) continue;
      int xn = x + cx[k], yn = y + cy[k];
      xn = xn < 0 ? xn + P.nx : (xn >= P.nx ? xn - P.nx : xn);
      yn = yn < 0 ? yn + P.ny : (yn >= P.ny ? yn - P.ny : yn);
      s += pl[ix(P, 1, 0, xn, yn)];
      ++c;
    }
    if (c > 0) {
      val = s / T(c);
      break;
    }
  }
  pl[ix(P, 1, 0, x, y)] = val;
}

// Field value at (x, y) of the extended grid x in [-1, nx], y in [-1, ny], as
// the stencils see it: x sides first, then y sides over the extended x range
// (corners take the y rule applied to the x ghosts).  Periodic sides wrap;
// walls take the wetting ghost of Eq. (50) (wet) or the mirror value.
template <typename T>
__device__ __forceinline__ T obs_pad_x(const Phys<T>& P, const T* pl, int x, int y, bool wet) {
  if (x >= 0 && x < P.nx) return pl[ix(P, 1, 0, x, y)];
  if (!P.wall_x) return pl[ix(P, 1, 0, x < 0 ? x + P.nx : x - P.nx, y)];
  if (x < 0) {
    const T c0 = pl[ix(P, 1, 0, 0, y)];
    return wet ? wall_ghost(P, SIDE_LEFT, c0, pl[ix(P, 1, 0, 1, y)]) : c0;
  }
  const T e0 = pl[ix(P, 1, 0, P.nx - 1, y)];
  return wet ? wall_ghost(P, SIDE_RIGHT, e0, pl[ix(P, 1, 0, P.nx - 2, y)]) : e0;
}
template <typename T>
__device__ __forceinline__ T obs_pad(const Phys<T>& P, const T* pl, int x, int y, bool wet) {
  if (y >= 0 && y < P.ny) return obs_pad_x(P, pl, x, y, wet);
  if (!P.wall_y) return obs_pad_x(P, pl, x, y < 0 ? y + P.ny : y - P.ny, wet);
  if (y < 0) {
    const T a = obs_pad_x(P, pl, x, 0, wet);
    return wet ? wall_ghost(P, SIDE_BOTTOM, a, obs_pad_x(P, pl, x, 1, wet)) : a;
  }
  const T a = obs_pad_x(P, pl, x, P.ny - 1, wet);
  return wet ? wall_ghost(P, SIDE_TOP, a, obs_pad_x(P, pl, x, P.ny - 2, wet)) : a;
}
// values at x + c_i, i = 0..8 (D2Q9 order)
template <typename T>
__device__ __forceinline__ void obs_gather9(const Phys<T>& P, const T* pl, int x, int y, bool wet, T v[9]) {
  if (x > 0 && x < P.nx - 1 && y > 0 && y < P.ny - 1) {
    const T* c = pl + ix(P, 1, 0, x, y);
    const long long r = P.pitch;
    v[0] = c[0];
    v[1] = c[1];
    v[2] = c[r];
    v[3] = c[-1];
    v[4] = c[-r];
    v[5] = c[r + 1];
    v[6] = c[r - 1];
    v[7] = c[-r - 1];
    v[8] = c[-r + 1];
    return;
  }
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int i = 0; i < 9; ++i) v[i] = obs_pad(P, pl, x + cx[i], y + cy[i], wet);
}

// Cahn-Hilliard: mu_phi (Eq. (5)) at the fluid nodes of [x_lo, x_hi) x
// [y_lo, y_lo + gridDim.y) from the filled phi plane (the Laplacian of Eq.
// (C.10) in the fused kernels' order); solid nodes are left to k_obs_fill.
template <typename T>
__global__ void k_obs_mu(const Phys<T> P, const T* __restrict__ phis, T* __restrict__ mus, int x_lo, int x_hi,
                         int y_lo) {
  // as k_obs_fill: let the next kernel start, wait for the phi plane
  asm volatile("griddepcontrol.launch_dependents;");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int x = x_lo + blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y_lo + blockIdx.y;
  if (x >= x_hi) return;
  if ((P.obs[(long long)y * P.nx + x] >> OBS_SOLID) & 1u) return;  // filled by k_obs_fill
  T p[9];
  obs_gather9(P, phis, x, y, true, p);
  const T ph = p[0];
  const T lap = (((p[1] - ph) + (p[3] - ph)) + ((p[2] - ph) + (p[4] - ph))) * T(2.0 / 3.0) +
                (((p[5] - ph) + (p[7] - ph)) + ((p[6] - ph) + (p[8] - ph))) * T(1.0 / 6.0);
  mus[ix(P, 1, 0, x, y)] = P.beta4 * (ph - P.phiA) * (ph - P.phiB) * (ph - P.phibar) - P.kappa * lap;
}

// Node update of every node in a mode; solid nodes write zeros.  One node
// per thread, so latency is hidden by residency alone: 8 blocks (32 warps)
// per SM, 64 registers (measured 8.2 against 7.2 GLUPS at 6 blocks on the
// 4096 x 2048 dam break over the obstacle, FP32).
template <class C, int MODEL, int MODE, bool UR>
__global__ void __launch_bounds__(OBS_THREADS, 8) k_obs_node(const Phys<typename C::value_t> P,
                                                         const Bufs<typename C::value_t> B,
                                                         const typename C::value_t* __restrict__ phis,
                                                         const typename C::value_t* __restrict__ mus) {
  using T = typename C::value_t;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  const long long pc = P.pitch;
  const unsigned m = P.obs[(long long)y * P.nx + x];
  if ((m >> OBS_SOLID) & 1u) {
    const T z[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    using CS = typename std::conditional<MODE == MODE_INIT, PopPlain<T>, C>::type;
    if (MODE == MODE_STEP || MODE == MODE_INIT) {
      store_pops<CS>(P, B.fout, 0, x, y, z, T(0), true);
      store_pops<CS>(P, B.gout, 1, x, y, z, T(0), false);
    }
    if (MODE == MODE_STEP || MODE == MODE_HIST) {
      T* hb = B.hist + ix(P, 5, 0, x, y);
#pragma unroll
      for (int k = 0; k < 5; ++k) hb[k * pc] = T(0);
      if (B.phi_prev) B.phi_prev[ix(P, 1, 0, x, y)] = T(0);
    }
    if (MODE == MODE_MACRO) {
      T* M = B.macro + ix(P, NMACRO, 0, x, y);
      for (int k = 0; k < NMACRO; ++k) M[k * pc] = T(0);
    }
    return;
  }
  T phi9[9], mu9[9];
  obs_gather9(P, phis, x, y, true, phi9);
  if (MODEL == MODEL_CH) obs_gather9(P, mus, x, y, false, mu9);
  T f[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T g[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  T h[5] = {T(0), T(0), T(0), T(0), T(0)};
  T uin = T(0), vin = T(0), pin = T(0);
  if (MODE == MODE_INIT) {
    const long long di = (long long)y * P.nx + x;
    if (B.iux) uin = T(B.iux[di]);
    if (B.iuy) vin = T(B.iuy[di]);
    if (B.ip) pin = T(B.ip[di]);
  } else {
    if (MODE == MODE_STEP) pull9_obs<C>(B.fin, P, 0, x, y, m, f);
    pull9_obs<C>(B.gin, P, 1, x, y, m, g);
    if (MODE == MODE_STEP || MODE == MODE_MACRO) {
#pragma unroll
      for (int k = 0; k < 5; ++k) h[k] = B.hist[ix(P, 5, k, x, y)];
    }
  }
  node_update<C, MODEL, MODE, UR>(P, B, x, y, phi9, mu9, f, g, h, uin, vin, pin);
}

}  // namespace pflbm
