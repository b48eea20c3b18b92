// Device code of the GB300 phase-field lattice Boltzmann path.
//
// Method: Zhan, Chai & Shi, "Consistent and conservative phase-field based
// lattice Boltzmann method for incompressible two-phase flows"
// (arXiv:2111.00847), Sec. 3 and App. C.  One launch of k_march<T, MODEL,
// MODE_STEP> advances the whole grid by one time step.
//
// Memory layout (HBM).  Populations are structure-of-arrays planes, one per
// D2Q9 direction, interleaved by rows: element i of node (x, y) of a set of
// NP planes sits at (y NP + i) pitch + XPAD + x (x fastest, pitch a multiple
// of 32 elements).  The nine plane-rows of a grid row are thus one pitch
// apart, so a node's nine stores share one base address with immediate
// offsets, and a row of all planes is one contiguous block.  There are two
// copies (A/B) of each population set.  A plane holds
// the POST-COLLISION value of each node (what it sends); the next step pulls
// f_i(x) = f_i*(x - c_i) from it, or the reflected f_{opp(i)}*(x) where
// x - c_i lies beyond a half-way bounce-back wall.  The hydrodynamic g_0 is
// stored minus the constant rho0 of Eq. (19): rho0 is an eigen-direction of
// the collision (M (rho0 e_0) = rho0 (1,-4,4,0,...)), so it passes through
// unchanged and only costs FP32 precision if kept in g_0.  Five history
// planes hold chi(t-1) for the explicit-Euler time derivatives of App. C.
//
// Kernel shape (k_march).  A block of BX threads owns an x-strip of BX
// columns and marches up a y-segment of LY rows; one thread per column.
// phi = sum_i f_i of a row is formed once, from the pulled populations the
// thread keeps in registers for that row's collision one (AC) or two (CH)
// iterations later, and parked in a shared-memory ring of rows, so the
// isotropic stencils read every phi from shared memory; the only redundant
// global traffic is the two halo columns per row (L2 hits: the neighbouring
// strips march alongside) and the R look-ahead rows at each segment start.
// Per lattice update the kernel reads 18 populations + 5 history values and
// writes the same: 46 values, the algorithmic minimum of a fused step.
//
// No tensor cores: the step is a bandwidth-bound stencil with ~500 flops per
// node and no dense contraction.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>
#include <type_traits>

namespace pflbm {

enum { MODEL_AC = 0, MODEL_CH = 1 };
// k_march modes:
//  STEP : pull, collide, store populations + history (+ phi(t) when asked)
//  MACRO: pull, write the macroscopic fields of time t (no state change)
//  HIST : pull, write the history chi(t) only (set-up after init / resume)
//  INIT : phi, u, p from device doubles; write f^eq, g^eq per node
enum { MODE_STEP = 0, MODE_MACRO = 1, MODE_HIST = 2, MODE_INIT = 3 };
enum {
  MAC_PHI = 0, MAC_UX, MAC_UY, MAC_P, MAC_RHO, MAC_MU, MAC_MCX, MAC_MCY, MAC_TRS, NMACRO
};
enum { SIDE_LEFT = 0, SIDE_RIGHT = 1, SIDE_BOTTOM = 2, SIDE_TOP = 3 };

constexpr int BX = 128;  // threads per block = columns per strip
constexpr int LY = 64;   // rows per block
constexpr int RING = 8;  // shared-memory ring of phi rows (power of two)
// Each stored row has XPAD pad elements on either side of its nx nodes
// (x in [-XPAD, nx + XPAD)).
// With a periodic x boundary the pads of the population planes hold copies
// of the XPAD nodes at the opposite edge (written together with the nodes),
// so a 16-byte aligned bulk copy of [x0 - XPAD, x0 + BX + XPAD) of a row
// carries its own halo.
constexpr int XPAD = 4;

// Per-run constants, in the arithmetic type.
template <typename T>
struct Phys {
  int nx, ny, pitch;
  long long plane;  // ny * pitch: elements per plane
  int wall_x, wall_y;
  int gravity_mode, visc_inverse, sg7_node, sg8_node;
  T phiA, phiB, phibar, inv_dphi;
  T beta4, kappa, lam_coef;  // 4 beta, k, sqrt(2 beta / k)   (Eqs. (3), (5), (8))
  T n_delta;                 // regularisation of |grad phi| in n = grad phi / |grad phi|
  T drho, rhoB, rho_mean;    // d rho / d phi, rho_B, (rho_A + rho_B)/2
  T mob_drho;                // (d rho/d phi) M_phi, zero for the original model
  T muA, muB, inuA, inuB;    // mu_A, mu_B, 1/nu_A, 1/nu_B
  T gx, gy, eta, H, K;
  T sf[9], hf[9];            // s_f^k and 1 - s_f^k / 2
  T sg[9], hg[9];
  T wa[4];                   // a = 4 cos(theta) / (W dphi) per side, Eq. (50)
  // 16-bit deviation storage (PopDev): per population set (0 = f, 1 = g)
  // the reference ratios r (axis, diagonal directions), the power-of-two
  // scale s of the stored deviations and 1/s, and for f the factor
  // 1 / (1 + sum_i r_i) that makes a node's decoded populations sum to phi.
  T dv_r[2][2], dv_s[2], dv_is[2], dv_c0;
  int seg_rows;  // rows per block segment of the TMA step on small grids (set by its launcher)
  int diag_y0, diag_y1;  // rows [diag_y0, diag_y1) enter the diagnostics (a y-slab: its own rows)
  // Solid obstacles (nullptr: none).  Per node of the dense [ny][nx] grid:
  // bit i-1 (i = 1..8) set when link i reflects, i.e. its upstream node
  // x - c_i is solid or lies beyond a wall; bit OBS_SOLID set at solid nodes.
  const uint16_t* obs;
  // solid nodes with a fluid node among their 8 neighbours (dense indices
  // y * nx + x): the only solid nodes a fluid stencil reads
  const int* obs_fill;
  int obs_nfill;
  // per block of the TMA step's launch grid (Allen-Cahn or Cahn-Hilliard):
  // nonzero when a solid node lies within 3 nodes of the block's rows and
  // columns (nullptr: every block); blocks away from obstacles take the
  // plain step's path
  const uint8_t* obs_near;
  int obs_box[4];     // x_lo, x_hi, y_lo, y_hi: the region of the phi plane the passes fill for them
  int obs_box_mu[4];  // the same for the mu_phi plane (Cahn-Hilliard)
};
constexpr int OBS_SOLID = 8;

// Population sets are addressed in bytes through a storage codec: plane 0
// of a row block holds B0-byte elements, planes 1..8 BI-byte elements, and
// a row block is pitch (B0 + 8 BI) bytes.  PopPlain stores every population
// in the arithmetic type (the layout in the file header).  PopDev<Q> stores
// the rest population f_0 (g_0) of a node in FP32 and the eight moving ones
// as Q (FP16 or BF16) deviations from r_i times it:
//   q_i = Q( s (f_i - r_i f_0) ),   decoded  f_i = q_i / s + r_i f_0,
// where r_i is the ratio f_i / f_0 of the node at rest, so that q_i carries
// only the velocity and non-equilibrium part.  For f the stored f_0 is then
// re-solved from the rounded q_i so that the decoded nine sum to phi
// exactly (conservation of phi does not depend on the 16-bit rounding).
template <typename T>
struct PopPlain {
  using value_t = T;
  using raw_t = T;
  static constexpr bool dev = false;
  static constexpr int B0 = sizeof(T), BI = sizeof(T);
};
template <typename Q>
struct PopDev {
  using value_t = float;
  using raw_t = Q;
  static constexpr bool dev = true;
  static constexpr int B0 = 4, BI = 2;
};
template <class C>
__host__ __device__ constexpr long long pop_row_bytes(long long pitch) {
  return pitch * (C::B0 + 8 * C::BI);
}
template <class C>
__host__ __device__ constexpr long long pop_plane_off(long long pitch, int i) {
  return i == 0 ? 0 : pitch * (C::B0 + (i - 1) * C::BI);
}

__device__ __forceinline__ uint16_t enc16(__half, float v) { return __half_as_ushort(__float2half_rn(v)); }
__device__ __forceinline__ uint16_t enc16(__nv_bfloat16, float v) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float dec16(__half, uint16_t q) { return __half2float(__ushort_as_half(q)); }
__device__ __forceinline__ float dec16(__nv_bfloat16, uint16_t q) {
  return __bfloat162float(__ushort_as_bfloat16(q));
}
// q * s + c in one mixed-precision FMA (16-bit q and s, FP32 c and result).
// With s a power of two that Q holds exactly, q * s is exact and this equals
// fmaf(dec16(q), float(s), c) bit for bit, without the separate conversion.
__device__ __forceinline__ float fma16(__half, uint16_t q, uint16_t s, float c) {
  float d;
  asm("fma.rn.f32.f16 %0, %1, %2, %3;" : "=f"(d) : "h"(q), "h"(s), "f"(c));
  return d;
}
__device__ __forceinline__ float fma16(__nv_bfloat16, uint16_t q, uint16_t s, float c) {
  float d;
  asm("fma.rn.f32.bf16 %0, %1, %2, %3;" : "=f"(d) : "h"(q), "h"(s), "f"(c));
  return d;
}

template <typename T>
struct Bufs {
  const void* fin;  // population set (codec layout), post-collision f of t-1
  const void* gin;
  void* fout;       // STEP: post-collision f of t;  INIT: f^eq per node (plain)
  void* gout;
  T* hist;        // 5 interleaved planes
  T* macro;       // NMACRO interleaved planes (MACRO)
  T* phi_prev;    // optional: phi(t) of the stepped time (STEP / HIST)
  const T* phis;  // solid obstacles: phi with the neutral-wetting fill (one plane)
  const T* mus;   // solid obstacles, Cahn-Hilliard: mu_phi with the fill (one plane)
  const double* iphi;  // INIT inputs, dense [ny][nx]
  const double* iux;
  const double* iuy;
  const double* ip;
};

__host__ __device__ constexpr int slot_of(int r) { return (r + 2 * RING) & (RING - 1); }

// Division and the normal's 1/(|grad phi|^4 + delta^4)^(1/4): IEEE in FP64
// (the path held to 1e-12 against the oracle), hardware approximations in
// FP32 (<= 2 ulp each, far inside the FP32 tolerance) where they save the
// slow path of an IEEE divide or square root.
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double inv_soft_norm(double g2, double delta) {
  const double d2 = delta * delta;
  return 1.0 / sqrt(sqrt(g2 * g2 + d2 * d2));
}
__device__ __forceinline__ float inv_soft_norm(float g2, float delta) {
  // S^(-1/4) = y * y^(-1/2) with y = S^(-1/2): two reciprocal square roots
  const float d2 = delta * delta;
  const float y = rsqrtf(g2 * g2 + d2 * d2);
  return y * rsqrtf(y);
}

// element k of a set of NP row-interleaved planes at node (x, y)
template <typename T>
__device__ __forceinline__ long long ix(const Phys<T>& P, int NP, int k, int x, int y) {
  return ((long long)y * NP + k) * P.pitch + XPAD + x;
}

// Decoded population i of node (x, r) of a set in codec C's layout.
template <class C>
__device__ __forceinline__ typename C::value_t pop_ld(const unsigned char* __restrict__ buf,
                                                      const Phys<typename C::value_t>& P, int set, int i,
                                                      int x, int r) {
  using T = typename C::value_t;
  const unsigned char* rb = buf + (long long)r * pop_row_bytes<C>(P.pitch);
  if constexpr (!C::dev) {
    return reinterpret_cast<const T*>(rb)[(long long)i * P.pitch + XPAD + x];
  } else {
    const float b = reinterpret_cast<const float*>(rb)[XPAD + x];
    if (i == 0) return b;
    const uint16_t q = reinterpret_cast<const uint16_t*>(rb + pop_plane_off<C>(P.pitch, i))[XPAD + x];
    return fmaf(dec16(typename C::raw_t(), q), P.dv_is[set], P.dv_r[set][i >= 5] * b);
  }
}

// ---------------------------------------------------------------------------
// Pull the nine populations of node (x, r) from the post-collision planes,
// with periodic wrap or half-way bounce-back at walls (Sec. 4).
// ---------------------------------------------------------------------------
template <class C>
__device__ __forceinline__ void pull9(const void* buf_, const Phys<typename C::value_t>& P, int set, int x,
                                      int r, typename C::value_t out[9]) {
  using T = typename C::value_t;
  int xm = x - 1, xp = x + 1, ym = r - 1, yp = r + 1;
  bool bxm = false, bxp = false, bym = false, byp = false;
  if (xm < 0) { if (P.wall_x) bxm = true; else xm += P.nx; }
  if (xp >= P.nx) { if (P.wall_x) bxp = true; else xp -= P.nx; }
  if (ym < 0) { if (P.wall_y) bym = true; else ym += P.ny; }
  if (yp >= P.ny) { if (P.wall_y) byp = true; else yp -= P.ny; }
  if constexpr (!C::dev) {
    const T* buf = static_cast<const T*>(buf_);
    const long long pl = P.pitch;  // plane i of a row sits i * pitch after plane 0
    const long long rc = (long long)r * 9 * pl + XPAD, rm = (long long)ym * 9 * pl + XPAD,
                    rp = (long long)yp * 9 * pl + XPAD;
    const long long c = rc + x;
    out[0] = buf[c];
    out[1] = buf[bxm ? 3 * pl + c : 1 * pl + rc + xm];
    out[2] = buf[bym ? 4 * pl + c : 2 * pl + rm + x];
    out[3] = buf[bxp ? 1 * pl + c : 3 * pl + rc + xp];
    out[4] = buf[byp ? 2 * pl + c : 4 * pl + rp + x];
    out[5] = buf[(bxm || bym) ? 7 * pl + c : 5 * pl + rm + xm];
    out[6] = buf[(bxp || bym) ? 8 * pl + c : 6 * pl + rm + xp];
    out[7] = buf[(bxp || byp) ? 5 * pl + c : 7 * pl + rp + xp];
    out[8] = buf[(bxm || byp) ? 6 * pl + c : 8 * pl + rp + xm];
  } else {
    const unsigned char* buf = static_cast<const unsigned char*>(buf_);
    out[0] = pop_ld<C>(buf, P, set, 0, x, r);
    out[1] = bxm ? pop_ld<C>(buf, P, set, 3, x, r) : pop_ld<C>(buf, P, set, 1, xm, r);
    out[2] = bym ? pop_ld<C>(buf, P, set, 4, x, r) : pop_ld<C>(buf, P, set, 2, x, ym);
    out[3] = bxp ? pop_ld<C>(buf, P, set, 1, x, r) : pop_ld<C>(buf, P, set, 3, xp, r);
    out[4] = byp ? pop_ld<C>(buf, P, set, 2, x, r) : pop_ld<C>(buf, P, set, 4, x, yp);
    out[5] = (bxm || bym) ? pop_ld<C>(buf, P, set, 7, x, r) : pop_ld<C>(buf, P, set, 5, xm, ym);
    out[6] = (bxp || bym) ? pop_ld<C>(buf, P, set, 8, x, r) : pop_ld<C>(buf, P, set, 6, xp, ym);
    out[7] = (bxp || byp) ? pop_ld<C>(buf, P, set, 5, x, r) : pop_ld<C>(buf, P, set, 7, xp, yp);
    out[8] = (bxm || byp) ? pop_ld<C>(buf, P, set, 6, x, r) : pop_ld<C>(buf, P, set, 8, xm, yp);
  }
}

// The same pull on a grid with solid obstacles, given the node's link word
// m (P.obs): a flagged link reflects (half-way bounce-back at the solid
// surface, as at a wall); a solid node sees no populations.  The nine
// streamed loads are issued first, from wrapped (always in-grid) upstream
// nodes, so that their addresses do not wait for m; the reflected links are
// then reloaded, which only nodes next to a boundary do.
template <class C>
__device__ __forceinline__ void pull9_obs(const void* buf_, const Phys<typename C::value_t>& P, int set, int x,
                                          int r, unsigned m, typename C::value_t out[9]) {
  using T = typename C::value_t;
  const unsigned char* buf = static_cast<const unsigned char*>(buf_);
  constexpr int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  constexpr int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  constexpr int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int sx = x - cx[i], sy = r - cy[i];
    sx = sx < 0 ? sx + P.nx : (sx >= P.nx ? sx - P.nx : sx);
    sy = sy < 0 ? sy + P.ny : (sy >= P.ny ? sy - P.ny : sy);
    out[i] = pop_ld<C>(buf, P, set, i, sx, sy);
  }
  if (m & 0x1ffu) {
    if ((m >> OBS_SOLID) & 1u) {
#pragma unroll
      for (int i = 0; i < 9; ++i) out[i] = T(0);
      return;
    }
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if ((m >> (i - 1)) & 1u) out[i] = pop_ld<C>(buf, P, set, op[i], x, r);
  }
}
template <class C>
__device__ __forceinline__ void pull9_obs(const void* buf_, const Phys<typename C::value_t>& P, int set, int x,
                                          int r, typename C::value_t out[9]) {
  pull9_obs<C>(buf_, P, set, x, r, (unsigned)P.obs[(long long)r * P.nx + x], out);
}

// Encode and store the nine post-collision populations v of node (x, y)
// into a set in codec C's layout, with the periodic copies in the row pads.
// m0: the zeroth moment the stored populations must reproduce (phi for f;
// used when conserve is set).
template <class C>
__device__ __forceinline__ void store_pops(const Phys<typename C::value_t>& P, void* buf_, int set, int x,
                                           int y, const typename C::value_t v[9], typename C::value_t m0,
                                           bool conserve) {
  using T = typename C::value_t;
  const long long pc = P.pitch;
  const bool pads = !P.wall_x && (x < XPAD || x >= P.nx - XPAD);
  const int off = x < XPAD ? P.nx : -P.nx;
  const bool both = x < XPAD && x >= P.nx - XPAD;  // grids narrower than 2 XPAD: both pads
  if constexpr (!C::dev) {
    T* const o = static_cast<T*>(buf_) + ix(P, 9, 0, x, y);
#pragma unroll
    for (int i = 0; i < 9; ++i) o[i * pc] = v[i];
    if (pads) {
#pragma unroll
      for (int i = 0; i < 9; ++i) o[i * pc + off] = v[i];
      if (both)
#pragma unroll
        for (int i = 0; i < 9; ++i) o[i * pc - P.nx] = v[i];
    }
  } else {
    using Q = typename C::raw_t;
    const float s = P.dv_s[set], is = P.dv_is[set];
    const float b = v[0];
    uint16_t q[9];
    float sq = 0.f;
    const uint16_t is16 = enc16(Q(), is);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      q[i] = enc16(Q(), (v[i] - P.dv_r[set][i >= 5] * b) * s);
      sq = fma16(Q(), q[i], is16, sq);
    }
    const float b0 = conserve ? P.dv_c0 * (m0 - sq) : b;
    unsigned char* const rb = static_cast<unsigned char*>(buf_) + (long long)y * pop_row_bytes<C>(pc);
    float* const o0 = reinterpret_cast<float*>(rb) + XPAD + x;
    uint16_t* const oq = reinterpret_cast<uint16_t*>(rb + pop_plane_off<C>(pc, 1)) + XPAD + x;
    *o0 = b0;
#pragma unroll
    for (int i = 1; i < 9; ++i) oq[(i - 1) * pc] = q[i];
    if (pads) {
      o0[off] = b0;
#pragma unroll
      for (int i = 1; i < 9; ++i) oq[(i - 1) * pc + off] = q[i];
      if (both) {
        o0[-P.nx] = b0;
#pragma unroll
        for (int i = 1; i < 9; ++i) oq[(i - 1) * pc - P.nx] = q[i];
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T sum9(const T v[9]) {
  return ((v[0] + (v[1] + v[3])) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
}

// phi of the in-domain node (x, r) in a given mode.
template <class C, int MODE, typename T = typename C::value_t>
__device__ __forceinline__ T phi_at(const Phys<T>& P, const Bufs<T>& B, int x, int r) {
  if (MODE == MODE_INIT) {
    return T(B.iphi[(long long)r * P.nx + x]);
  } else {
    T v[9];
    pull9<C>(B.fin, P, 0, x, r, v);
    return sum9(v);
  }
}

// Products and sums rounded one by one (never contracted into an FMA), so
// that every call site of a function built from them returns the same bits.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// Wetting ghost, Eqs. (49)-(50): phi_w is the root the paper selects,
// (-b + sqrt(b^2 - 4ac)) / (2a), evaluated as 2c / (-b - sqrt(b^2 - 4ac))
// (the same number; finite as a -> 0, where it tends to -c/b); the ghost at
// -1/2 is the quadratic through (0, phi_w), (1/2, phi_1), (3/2, phi_2).
// Every operation is rounded on its own: a kernel forms the ghost at more
// than one place (a segment's first row from global memory, the others from
// staged rows), and a grid divided into y-slabs must see the same value at
// either place.
template <typename T>
__device__ __forceinline__ T wall_ghost(const Phys<T>& P, int side, T phi1, T phi2) {
  const T a = P.wa[side];
  const T b = add_rn(T(8.0 / 3.0), -mul_rn(a, add_rn(P.phiA, P.phiB)));
  const T c = add_rn(add_rn(mul_rn(mul_rn(a, P.phiA), P.phiB), mul_rn(phi2, T(1.0 / 3.0))), -mul_rn(T(3), phi1));
  T disc = add_rn(mul_rn(b, b), -mul_rn(mul_rn(T(4), a), c));
  disc = disc > T(0) ? disc : T(0);
  const T phiw = mul_rn(T(2), c) / add_rn(-b, -sqrt(disc));
  return add_rn(add_rn(mul_rn(T(8.0 / 3.0), phiw), -mul_rn(T(2), phi1)), mul_rn(phi2, T(1.0 / 3.0)));
}

// ---------------------------------------------------------------------------
// Per-node update.  phi9 / mu9: values at x + c_i (D2Q9 order), f, g: pulled
// populations, h: chi(t-1).  Writes the outputs of the mode.
// ---------------------------------------------------------------------------
// UR ("unit rates"): the relaxation rates of Sec. 4 that the paper leaves at
// 1 are 1 (s_f^k for k != 3, 5 and s_g^k for k = 0, 1, 2, 3, 5); those
// moments then relax to m^eq + m_src / 2 without reading the populations'
// own moments, which the general path (UR = false) computes and relaxes.
// C: the storage codec of the STEP outputs (INIT writes plain values).
template <class C, int MODEL, int MODE, bool UR = false, typename T = typename C::value_t>
__device__ __forceinline__ void node_update(const Phys<T>& P, const Bufs<T>& B, int x, int y,
                                            const T phi9[9], const T mu9[9], const T f[9],
                                            const T g[9], const T h[5], T u_in, T v_in, T p_in) {
  const T phi = phi9[0];
  const long long pc = P.pitch;
  // isotropic gradient and Laplacian, Eqs. (C.9)-(C.10) (c_s^2 = 1/3):
  // grad = 3 sum w_i c_i phi_i ; lap = 6 sum w_i (phi_i - phi)
  const T gx = (phi9[1] - phi9[3]) * T(1.0 / 3.0) + ((phi9[5] - phi9[7]) + (phi9[8] - phi9[6])) * T(1.0 / 12.0);
  const T gy = (phi9[2] - phi9[4]) * T(1.0 / 3.0) + ((phi9[5] - phi9[7]) + (phi9[6] - phi9[8])) * T(1.0 / 12.0);
  T mu, Dx, Dy, lam = T(0), nnx = T(0), nny = T(0);
  if (MODEL == MODEL_AC) {
    // differences first: neighbouring phi are close, so phi_i - phi is exact
    const T lap = (((phi9[1] - phi) + (phi9[3] - phi)) + ((phi9[2] - phi) + (phi9[4] - phi))) * T(2.0 / 3.0) +
                  (((phi9[5] - phi) + (phi9[7] - phi)) + ((phi9[6] - phi) + (phi9[8] - phi))) * T(1.0 / 6.0);
    // chemical potential, Eq. (5)
    mu = P.beta4 * (phi - P.phiA) * (phi - P.phiB) * (phi - P.phibar) - P.kappa * lap;
    // conservative AC flux, Eqs. (7)-(8), n = grad phi / (|grad phi|^4 + delta_n^4)^(1/4)
    // (delta_n = n_delta dphi / W, default n_delta 5e-3: the unit normal across
    // the interface, and a smooth function of grad phi with slope about
    // 1/delta_n in the bulk, where |grad phi| -> 0)
    lam = P.lam_coef * (P.phiA - phi) * (phi - P.phiB);
    const T inv = inv_soft_norm(gx * gx + gy * gy, P.n_delta);
    nnx = gx * inv;
    nny = gy * inv;
    Dx = gx - lam * nnx;
    Dy = gy - lam * nny;
  } else {
    // CH: D = grad mu_phi (Eq. (6)), mu9 holds mu_phi at x + c_i
    mu = mu9[0];
    Dx = (mu9[1] - mu9[3]) * T(1.0 / 3.0) + ((mu9[5] - mu9[7]) + (mu9[8] - mu9[6])) * T(1.0 / 12.0);
    Dy = (mu9[2] - mu9[4]) * T(1.0 / 3.0) + ((mu9[5] - mu9[7]) + (mu9[6] - mu9[8])) * T(1.0 / 12.0);
  }
  // density (Eq. (10)), its gradient, consistent flux (Eq. (15)), force
  const T rho = P.drho * (phi - P.phiB) + P.rhoB;
  const T rx = P.drho * gx, ry = P.drho * gy;
  const T mcx = -P.mob_drho * Dx, mcy = -P.mob_drho * Dy;
  const T Gs = P.gravity_mode == 0 ? T(1) : (P.gravity_mode == 1 ? rho : rho - P.rho_mean);
  const T Fx = mu * gx + Gs * P.gx, Fy = mu * gy + Gs * P.gy;

  // zeroth- and first-order sums of g
  const T ga = (g[1] + g[3]) + (g[2] + g[4]);
  const T gb = (g[5] + g[7]) + (g[6] + g[8]);
  const T g13 = g[1] - g[3], g24 = g[2] - g[4];
  const T gdx = (g[5] - g[7]) + (g[8] - g[6]);
  const T gdy = (g[5] - g[7]) + (g[6] - g[8]);
  T u, v;
  if (MODE == MODE_INIT) {
    u = u_in;
    v = v_in;
  } else {
    // Eq. (22b): rho u = sum c_i g_i + F/2
    const T irho = fdiv(T(1), rho);
    u = ((g13 + gdx) + T(0.5) * Fx) * irho;
    v = ((g24 + gdy) + T(0.5) * Fy) * irho;
  }
  const T um = u * mcx + v * mcy;   // u . m
  const T cA = u * mcx - v * mcy;   // u m_x - v m_y
  const T cB = u * mcy + v * mcx;   // u m_y + v m_x
  const T phu = phi * u, phv = phi * v;
  T d_phu = T(0), d_phv = T(0), d_um = T(0), d_A = T(0), d_B = T(0);
  if (MODE == MODE_STEP || MODE == MODE_MACRO) {
    d_phu = phu - h[0];
    d_phv = phv - h[1];
    d_um = um - h[2];
    d_A = cA - h[3];
    d_B = cB - h[4];
  }
  const T uu = u * u + v * v;
  const T ugr = u * rx + v * ry;
  const T uF = u * Fx + v * Fy;
  T p;
  if (MODE == MODE_INIT) {
    p = p_in;
  } else {
    // Eq. (39), second way: s_0 = -w_0 (rho u.u + u.m)/(2 c_s^2) = -(2/3)(...)
    const T s0 = T(-2.0 / 3.0) * (rho * uu + um);
    p = T(0.6) * ((ga + gb) + (T(0.5) + P.H) * ugr + s0 + P.K * (T(2) * uF + d_um));
  }

  if (MODE == MODE_HIST || MODE == MODE_STEP) {
    {
      T* hb = B.hist + ix(P, 5, 0, x, y);
      hb[0] = phu;
      hb[pc] = phv;
      hb[2 * pc] = um;
      hb[3 * pc] = cA;
      hb[4 * pc] = cB;
    }
    if (B.phi_prev) B.phi_prev[ix(P, 1, 0, x, y)] = phi;
    if (MODE == MODE_HIST) return;
  }

  // viscous rate s_g^{7,8} = 1/(nu/c_s^2 + 1/2), nu from Eq. (11) or (12)
  T s7 = P.sg[7], s8 = P.sg[8];
  if (P.sg7_node | P.sg8_node) {
    const T frac = (phi - P.phiB) * P.inv_dphi;
    T snode;
    if (!P.visc_inverse) {
      const T muv = frac * (P.muA - P.muB) + P.muB;
      snode = fdiv(rho, T(3) * muv + T(0.5) * rho);
    } else {
      const T inu = frac * (P.inuA - P.inuB) + P.inuB;
      snode = fdiv(inu, T(3) + T(0.5) * inu);
    }
    if (P.sg7_node) s7 = snode;
    if (P.sg8_node) s8 = snode;
  }

  // hydrodynamic moments m = M g (deviation form: g_0 without rho0)
  const T m0 = g[0] + ga + gb;
  const T m1 = T(-4) * g[0] - ga + T(2) * gb;

  // equilibrium moments, Eq. (C.2), minus rho0 (1, -4, 4, 0, ...)
  const T E1 = T(6) * p + T(3) * (rho * uu + um);
  const T E2 = T(-9) * p - T(3) * (rho * uu + um);
  const T E3 = rho * u, E5 = rho * v;
  const T E7 = cA + rho * (u * u - v * v);
  const T E8 = T(0.5) * cB + rho * u * v;
  // forcing moments, Eq. (C.2)
  const T Q0 = ugr;
  const T Q1 = T(3) * d_um + T(6) * uF;
  const T Q2 = -ugr - Q1;
  const T Q7 = T(2.0 / 3.0) * (u * rx - v * ry) + T(2) * (u * Fx - v * Fy) + d_A;
  const T Q8 = T(1.0 / 3.0) * (u * ry + v * rx) + (u * Fy + v * Fx) + T(0.5) * d_B;

  if (MODE == MODE_MACRO) {
    // strain-rate trace, Eq. (35): tr S = -s_2/(2 rho c_s^2)[tr sum cc(g - g^eq) + tr M_2F / 2]
    const T trneq = ((m1 - E1) + T(4) * m0) * T(1.0 / 3.0);
    const T trM2F = (Q1 + T(4) * Q0) * T(1.0 / 3.0);
    const T trS = -s7 * T(1.5) / rho * (trneq + T(0.5) * trM2F);
    T* M = B.macro + ix(P, NMACRO, 0, x, y);
    M[MAC_PHI * pc] = phi;
    M[MAC_UX * pc] = u;
    M[MAC_UY * pc] = v;
    M[MAC_P * pc] = p;
    M[MAC_RHO * pc] = rho;
    M[MAC_MU * pc] = mu;
    M[MAC_MCX * pc] = mcx;
    M[MAC_MCY * pc] = mcy;
    M[MAC_TRS * pc] = trS;
    return;
  }

  // ---- phase-field collision, Eq. (17) with Eq. (C.4) (AC) / (C.3) (CH)
  const T chi = (MODEL == MODEL_AC) ? phi : mu;
  const T e1 = T(-4) * phi + T(2) * P.eta * chi;
  const T e2 = T(4) * phi - T(3) * P.eta * chi;
  T Xx = d_phu, Xy = d_phv;
  if (MODEL == MODEL_AC) {
    Xx += lam * nnx * T(1.0 / 3.0);
    Xy += lam * nny * T(1.0 / 3.0);
  }
  T fs[9];
  if (MODE == MODE_INIT) {
    // f^eq = M^{-1} m^eq
    const T a = phi * T(1.0 / 9.0) - e1 * T(1.0 / 36.0) - e2 * T(1.0 / 18.0);
    const T b = phi * T(1.0 / 9.0) + e1 * T(1.0 / 18.0) + e2 * T(1.0 / 36.0);
    const T X = phu * T(1.0 / 3.0), Y = phv * T(1.0 / 3.0);        // m3/6 - m4/6 with m4 = -m3
    const T Xd = phu * T(1.0 / 12.0), Yd = phv * T(1.0 / 12.0);    // m3/6 + m4/12
    fs[0] = (phi - e1 + e2) * T(1.0 / 9.0);
    fs[1] = a + X; fs[3] = a - X; fs[2] = a + Y; fs[4] = a - Y;
    fs[5] = b + Xd + Yd; fs[6] = b - Xd + Yd; fs[7] = b - Xd - Yd; fs[8] = b + Xd - Yd;
  } else if (UR) {
    // only j_x, j_y (moments 3, 5) relax at s_f^{3,5}; the others take
    // m^eq + m_R / 2 (m_R vanishes in moments 0-2, 7, 8)
    const T f13 = f[1] - f[3], f24 = f[2] - f[4];
    const T fdx = (f[5] - f[7]) + (f[8] - f[6]);
    const T fdy = (f[5] - f[7]) + (f[6] - f[8]);
    const T m3 = f13 + fdx, m5 = f24 + fdy;
    const T s3 = m3 + P.sf[3] * (phu - m3) + P.hf[3] * Xx;
    const T s5 = m5 + P.sf[5] * (phv - m5) + P.hf[5] * Xy;
    const T s4 = -phu - T(0.5) * Xx;
    const T s6 = -phv - T(0.5) * Xy;
    const T a = phi * T(1.0 / 9.0) - e1 * T(1.0 / 36.0) - e2 * T(1.0 / 18.0);
    const T b = phi * T(1.0 / 9.0) + e1 * T(1.0 / 18.0) + e2 * T(1.0 / 36.0);
    const T X = (s3 - s4) * T(1.0 / 6.0), Y = (s5 - s6) * T(1.0 / 6.0);
    const T Xd = s3 * T(1.0 / 6.0) + s4 * T(1.0 / 12.0);
    const T Yd = s5 * T(1.0 / 6.0) + s6 * T(1.0 / 12.0);
    fs[0] = (phi - e1 + e2) * T(1.0 / 9.0);
    fs[1] = a + X; fs[3] = a - X; fs[2] = a + Y; fs[4] = a - Y;
    fs[5] = b + Xd + Yd; fs[6] = b - Xd + Yd; fs[7] = b - Xd - Yd; fs[8] = b + Xd - Yd;
  } else {
    const T fa = (f[1] + f[3]) + (f[2] + f[4]);
    const T fb = (f[5] + f[7]) + (f[6] + f[8]);
    const T f13 = f[1] - f[3], f24 = f[2] - f[4];
    const T fdx = (f[5] - f[7]) + (f[8] - f[6]);
    const T fdy = (f[5] - f[7]) + (f[6] - f[8]);
    T m[9];
    m[0] = f[0] + fa + fb;
    m[1] = T(-4) * f[0] - fa + T(2) * fb;
    m[2] = T(4) * f[0] - T(2) * fa + fb;
    m[3] = f13 + fdx;
    m[4] = T(-2) * f13 + fdx;
    m[5] = f24 + fdy;
    m[6] = T(-2) * f24 + fdy;
    m[7] = (f[1] + f[3]) - (f[2] + f[4]);
    m[8] = (f[5] + f[7]) - (f[6] + f[8]);
    const T eq[9] = {phi, e1, e2, phu, -phu, phv, -phv, T(0), T(0)};
    const T src[9] = {T(0), T(0), T(0), Xx, -Xx, Xy, -Xy, T(0), T(0)};
#pragma unroll
    for (int k = 0; k < 9; ++k) m[k] = m[k] + P.sf[k] * (eq[k] - m[k]) + P.hf[k] * src[k];
    const T a = m[0] * T(1.0 / 9.0) - m[1] * T(1.0 / 36.0) - m[2] * T(1.0 / 18.0);
    const T b = m[0] * T(1.0 / 9.0) + m[1] * T(1.0 / 18.0) + m[2] * T(1.0 / 36.0);
    const T X = (m[3] - m[4]) * T(1.0 / 6.0), Y = (m[5] - m[6]) * T(1.0 / 6.0);
    const T Xd = m[3] * T(1.0 / 6.0) + m[4] * T(1.0 / 12.0);
    const T Yd = m[5] * T(1.0 / 6.0) + m[6] * T(1.0 / 12.0);
    const T Pp = m[7] * T(0.25), Qq = m[8] * T(0.25);
    fs[0] = (m[0] - m[1] + m[2]) * T(1.0 / 9.0);
    fs[1] = a + X + Pp; fs[3] = a - X + Pp; fs[2] = a + Y - Pp; fs[4] = a - Y - Pp;
    fs[5] = b + Xd + Yd + Qq; fs[6] = b - Xd + Yd - Qq;
    fs[7] = b - Xd - Yd + Qq; fs[8] = b + Xd - Yd - Qq;
  }

  // ---- hydrodynamic collision, Eq. (40) with Eq. (C.2)
  T gs[9];
  {
    T m[9], eq[9], src[9];
    if (MODE == MODE_INIT) {
      m[0] = m[1] = m[2] = m[3] = m[4] = m[5] = m[6] = m[7] = m[8] = T(0);
    } else {
      m[0] = m0;
      m[1] = m1;
      m[2] = T(4) * g[0] - T(2) * ga + gb;
      m[3] = g13 + gdx;
      m[4] = T(-2) * g13 + gdx;
      m[5] = g24 + gdy;
      m[6] = T(-2) * g24 + gdy;
      m[7] = (g[1] + g[3]) - (g[2] + g[4]);
      m[8] = (g[5] + g[7]) - (g[6] + g[8]);
    }
    eq[0] = T(0); eq[1] = E1; eq[2] = E2; eq[3] = E3; eq[4] = -E3; eq[5] = E5; eq[6] = -E5;
    eq[7] = E7; eq[8] = E8;
    src[0] = Q0; src[1] = Q1; src[2] = Q2; src[3] = Fx; src[4] = -Fx; src[5] = Fy; src[6] = -Fy;
    src[7] = Q7; src[8] = Q8;
    if (MODE == MODE_INIT) {
#pragma unroll
      for (int k = 0; k < 9; ++k) m[k] = eq[k];
    } else if (UR) {
      // moments 0, 1, 2, 3, 5 relax at rate 1: m^eq + m_F / 2
#pragma unroll
      for (int k = 0; k < 6; ++k)
        if (k != 4) m[k] = eq[k] + T(0.5) * src[k];
      m[4] = m[4] + P.sg[4] * (eq[4] - m[4]) + P.hg[4] * src[4];
      m[6] = m[6] + P.sg[6] * (eq[6] - m[6]) + P.hg[6] * src[6];
      m[7] = m[7] + s7 * (eq[7] - m[7]) + (T(1) - T(0.5) * s7) * src[7];
      m[8] = m[8] + s8 * (eq[8] - m[8]) + (T(1) - T(0.5) * s8) * src[8];
    } else {
#pragma unroll
      for (int k = 0; k < 7; ++k) m[k] = m[k] + P.sg[k] * (eq[k] - m[k]) + P.hg[k] * src[k];
      m[7] = m[7] + s7 * (eq[7] - m[7]) + (T(1) - T(0.5) * s7) * src[7];
      m[8] = m[8] + s8 * (eq[8] - m[8]) + (T(1) - T(0.5) * s8) * src[8];
    }
    const T a = m[0] * T(1.0 / 9.0) - m[1] * T(1.0 / 36.0) - m[2] * T(1.0 / 18.0);
    const T b = m[0] * T(1.0 / 9.0) + m[1] * T(1.0 / 18.0) + m[2] * T(1.0 / 36.0);
    const T X = (m[3] - m[4]) * T(1.0 / 6.0), Y = (m[5] - m[6]) * T(1.0 / 6.0);
    const T Xd = m[3] * T(1.0 / 6.0) + m[4] * T(1.0 / 12.0);
    const T Yd = m[5] * T(1.0 / 6.0) + m[6] * T(1.0 / 12.0);
    const T Pp = m[7] * T(0.25), Qq = m[8] * T(0.25);
    gs[0] = (m[0] - m[1] + m[2]) * T(1.0 / 9.0);
    gs[1] = a + X + Pp; gs[3] = a - X + Pp; gs[2] = a + Y - Pp; gs[4] = a - Y - Pp;
    gs[5] = b + Xd + Yd + Qq; gs[6] = b - Xd + Yd - Qq;
    gs[7] = b - Xd - Yd + Qq; gs[8] = b + Xd - Yd - Qq;
  }

  using CS = typename std::conditional<MODE == MODE_INIT, PopPlain<T>, C>::type;
  store_pops<CS>(P, B.fout, 0, x, y, fs, phi, true);
  store_pops<CS>(P, B.gout, 1, x, y, gs, T(0), false);
}

// ---------------------------------------------------------------------------
// The fused marching kernel.
// ---------------------------------------------------------------------------
template <class C, int MODEL, int MODE>
__global__ void __launch_bounds__(BX) k_march(const Phys<typename C::value_t> P,
                                              const Bufs<typename C::value_t> B) {
  using T = typename C::value_t;
  constexpr int R = (MODEL == MODEL_CH) ? 2 : 1;  // phi halo radius
  constexpr int WS = BX + 2 * R;                  // phi ring row width
  __shared__ T sphi[RING][WS];
  __shared__ T smu[(MODEL == MODEL_CH) ? RING : 1][BX + 2];

  const int tid = threadIdx.x;
  const int nx = P.nx, ny = P.ny;
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * LY;
  const int w = min(BX, nx - x0);
  const int y1 = min(y0 + LY, ny);
  const bool active = tid < w;
  const int x = x0 + tid;
  const bool left_edge = (x0 == 0), right_edge = (x0 + w == nx);
  const bool halo_l = (tid == 0), halo_r = (tid == w - 1);

  // Pulled populations of the rows not yet processed (look-ahead queue).
  T fq[R + 1][9];

  // -- make phi of row r (in-domain or periodic wrap) into the ring: own
  //    column, and the halo columns (threads 0 and w-1).  x-wall ghosts are
  //    computed by the halo threads from their own values (no barrier).
  auto make_row = [&](int r, int q) {
    int rr = r;
    if (rr < 0) rr += ny;
    if (rr >= ny) rr -= ny;
    const int s = slot_of(r);
    if (active) {
      T v;
      if (MODE == MODE_INIT) {
        v = T(B.iphi[(long long)rr * nx + x]);
      } else {
        pull9<C>(B.fin, P, 0, x, rr, fq[q]);
        v = sum9(fq[q]);
      }
      sphi[s][tid + R] = v;
      if (halo_l) {
#pragma unroll
        for (int k = 1; k <= R; ++k) {
          int xh = x0 - k;
          T hv;
          if (xh >= 0) {
            hv = phi_at<C, MODE>(P, B, xh, rr);
          } else if (!P.wall_x) {
            hv = phi_at<C, MODE>(P, B, xh + nx, rr);
          } else {  // ghost beyond the left wall, from columns 0 and 1
            const T p1 = (x == 0) ? v : phi_at<C, MODE>(P, B, 0, rr);
            hv = wall_ghost(P, SIDE_LEFT, p1, phi_at<C, MODE>(P, B, 1, rr));
          }
          sphi[s][R - k] = hv;
        }
      }
      if (halo_r) {
#pragma unroll
        for (int k = 1; k <= R; ++k) {
          int xh = x0 + w - 1 + k;
          T hv;
          if (xh < nx) {
            hv = phi_at<C, MODE>(P, B, xh, rr);
          } else if (!P.wall_x) {
            hv = phi_at<C, MODE>(P, B, xh - nx, rr);
          } else {  // ghost beyond the right wall, from columns nx-1 and nx-2
            const T p1 = (x == nx - 1) ? v : phi_at<C, MODE>(P, B, nx - 1, rr);
            hv = wall_ghost(P, SIDE_RIGHT, p1, phi_at<C, MODE>(P, B, nx - 2, rr));
          }
          sphi[s][w - 1 + R + k] = hv;
        }
      }
    }
  };
  // -- y-wall ghost row from two in-domain rows (after a barrier)
  auto ghost_row = [&](int r_ghost, int r1, int r2, int side) {
    const int sg = slot_of(r_ghost), s1 = slot_of(r1), s2 = slot_of(r2);
    for (int j = tid; j < w + 2 * R; j += BX) sphi[sg][j] = wall_ghost(P, side, sphi[s1][j], sphi[s2][j]);
  };
  // -- CH: mu_phi of row r over columns [-1, w] into the mu ring
  auto make_mu = [&](int r) {
    if (MODEL != MODEL_CH) return;
    const int s = slot_of(r);
    const int sm = slot_of(r - 1), sp = slot_of(r + 1);
    for (int j = tid - 1; j <= w; j += BX) {
      const int c = j + R;
      const T ph = sphi[s][c];
      const T lap = (((sphi[s][c + 1] - ph) + (sphi[s][c - 1] - ph)) + ((sphi[sp][c] - ph) + (sphi[sm][c] - ph))) *
                        T(2.0 / 3.0) +
                    (((sphi[sp][c + 1] - ph) + (sphi[sm][c - 1] - ph)) + ((sphi[sp][c - 1] - ph) + (sphi[sm][c + 1] - ph))) *
                        T(1.0 / 6.0);
      smu[s][j + 1] = P.beta4 * (ph - P.phiA) * (ph - P.phiB) * (ph - P.phibar) - P.kappa * lap;
    }
  };
  // -- CH: mirror ghosts of mu (x walls after make_mu, y walls whole rows)
  auto mu_xmirror = [&](int r) {
    if (MODEL != MODEL_CH || !P.wall_x) return;
    const int s = slot_of(r);
    if (left_edge && tid == 0) smu[s][0] = smu[s][1];
    if (right_edge && tid == 0) smu[s][w + 1] = smu[s][w];
  };
  auto mu_row_copy = [&](int r_dst, int r_src) {
    const int sd = slot_of(r_dst), ss = slot_of(r_src);
    for (int j = tid; j < w + 2; j += BX) smu[sd][j] = smu[ss][j];
  };

  const bool wy = P.wall_y != 0;

  // ------------------------------------------------------------ prologue
  // AC: rows y0-1, y0 (keep f of y0).  CH: rows y0-2 .. y0+1 (keep y0, y0+1).
#pragma unroll
  for (int k = -R; k <= R - 1; ++k) {
    const int r = y0 + k;
    const bool in = (r >= 0 && r < ny);
    if (in || !wy) make_row(r, k >= 0 ? k : 0);
  }
  __syncthreads();
  if (R == 2 && wy) {
    // CH look-ahead reaches a wall inside the prologue: the bottom ghost
    // needs rows 0 and 1, the top ghost (segment starting at ny-1) rows
    // ny-1 and ny-2 -- all made above.  (AC makes these ghosts in the march.)
    if (y0 == 0) {
      ghost_row(-1, 0, 1, SIDE_BOTTOM);
      __syncthreads();
    }
    if (y0 + R - 1 >= ny) {
      ghost_row(ny, ny - 1, ny - 2, SIDE_TOP);
      __syncthreads();
    }
  }
  if (MODEL == MODEL_CH) {
    // mu of rows y0-1 and y0
    if (wy && y0 == 0) {
      make_mu(0);
      __syncthreads();
      mu_xmirror(0);
      __syncthreads();
      mu_row_copy(-1, 0);
    } else {
      make_mu(y0 - 1);
      make_mu(y0);
      __syncthreads();
      mu_xmirror(y0 - 1);
      mu_xmirror(y0);
    }
    __syncthreads();
  }

  // ------------------------------------------------------------ march
  for (int y = y0; y < y1; ++y) {
    // make the look-ahead phi row y + R
    const int rn = y + R;
    const bool rn_in = rn < ny;
    if (rn_in || !wy) make_row(rn, R);
    // loads of the current row's g and history
    T g[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    T h[5] = {T(0), T(0), T(0), T(0), T(0)};
    T uin = T(0), vin = T(0), pin = T(0);
    if (active) {
      if (MODE == MODE_INIT) {
        const long long di = (long long)y * nx + x;
        if (B.iux) uin = T(B.iux[di]);
        if (B.iuy) vin = T(B.iuy[di]);
        if (B.ip) pin = T(B.ip[di]);
      } else {
        pull9<C>(B.gin, P, 1, x, y, g);
        if (MODE == MODE_STEP || MODE == MODE_MACRO) {
#pragma unroll
          for (int k = 0; k < 5; ++k) h[k] = B.hist[ix(P, 5, k, x, y)];
        }
      }
    }
    __syncthreads();
    if (wy) {
      if (R == 1 && y == 0) {  // bottom ghost now that row 1 exists
        ghost_row(-1, 0, 1, SIDE_BOTTOM);
        __syncthreads();
      }
      if (rn == ny) {  // top ghost from rows ny-1, ny-2
        ghost_row(ny, ny - 1, ny - 2, SIDE_TOP);
        __syncthreads();
      }
    }
    if (MODEL == MODEL_CH) {
      const int rm = y + 1;  // mu row needed next
      if (rm < ny || !wy) {
        make_mu(rm);
        __syncthreads();
        mu_xmirror(rm);
      } else if (rm == ny) {
        mu_row_copy(ny, ny - 1);
      }
      __syncthreads();
    }

    if (active) {
      const int sm = slot_of(y - 1), s0 = slot_of(y), sp = slot_of(y + 1);
      const int c = tid + R;
      T phi9[9];
      phi9[0] = sphi[s0][c];
      phi9[1] = sphi[s0][c + 1];
      phi9[2] = sphi[sp][c];
      phi9[3] = sphi[s0][c - 1];
      phi9[4] = sphi[sm][c];
      phi9[5] = sphi[sp][c + 1];
      phi9[6] = sphi[sp][c - 1];
      phi9[7] = sphi[sm][c - 1];
      phi9[8] = sphi[sm][c + 1];
      T mu9[9];
      if (MODEL == MODEL_CH) {
        const int cm = tid + 1;
        mu9[0] = smu[s0][cm];
        mu9[1] = smu[s0][cm + 1];
        mu9[2] = smu[sp][cm];
        mu9[3] = smu[s0][cm - 1];
        mu9[4] = smu[sm][cm];
        mu9[5] = smu[sp][cm + 1];
        mu9[6] = smu[sp][cm - 1];
        mu9[7] = smu[sm][cm - 1];
        mu9[8] = smu[sm][cm + 1];
      }
      node_update<C, MODEL, MODE>(P, B, x, y, phi9, mu9, fq[0], g, h, uin, vin, pin);
    }
    // advance the queue of pulled f
#pragma unroll
    for (int q = 0; q < R; ++q)
#pragma unroll
      for (int i = 0; i < 9; ++i) fq[q][i] = fq[q + 1][i];
  }
}

// ---------------------------------------------------------------------------
// TMA-staged fused step (Allen-Cahn, MODE_STEP): the hot path.
//
// Same per-node arithmetic as k_march, with the population rows brought in
// by the Tensor Memory Accelerator: one elected thread issues, per source
// row, nine 1-D bulk copies (cp.async.bulk) of the aligned segment
// [x0 - XPAD, x0 + BX + XPAD) of the f planes, and nine of the g planes, into
// shared-memory rings whose slots complete on an mbarrier (expect_tx bytes).
// Rows are requested one march step ahead, so the HBM latency of row y + 1
// overlaps the arithmetic of row y without holding the data in registers;
// the pull shifts become shared-memory index offsets and the halo columns
// arrive with the row.  Every wait is bounded: on time-out the block records
// the failure in *err (the host turns it into LBM_ECUDA), lets the copies it
// issued land (again with a bound) and returns.
//
// ---------------------------------------------------------------------------
// Staged columns per plane row, for a strip TBX wide.
template <int TBX>
struct Seg {
  static constexpr int value = TBX + 2 * XPAD;
};
// Rings: f rows y-1 .. y+2 are live while row y is processed (pulls of row y,
// phi of row y+1) and DF more rows are in flight; g rows y-1 .. y+1 are live
// and DG more are in flight.  SLIM: the pulled f of row y is kept in
// registers from phi's pass over that row, so f row y-1 is not needed and
// the f ring is one row shorter.
// phi ring of the TMA step: rows y-2 .. y+1 can be in use at once (slower
// threads of the previous march step read y-2 .. y while row y+1 is formed)
constexpr int TRING = 4;
__host__ __device__ constexpr int tslot(int r) { return (r + 2 * TRING) & (TRING - 1); }

// A staged row slot holds the segment of each of the nine planes: plane 0
// (SEG elements of B0 bytes) then planes 1..8 (SEG elements of BI bytes).
template <class C, int TBX, int DF, int DG, bool SLIM = false>
struct TmaLayout {
  using T = typename C::value_t;
  static constexpr int SEG = Seg<TBX>::value;
  static constexpr int RF = (SLIM ? 3 : 4) + DF, RG = 3 + DG;
  static constexpr size_t P0 = (size_t)SEG * C::B0;   // bytes of plane 0's segment
  static constexpr size_t PI = (size_t)SEG * C::BI;   // bytes of each other plane's segment
  static constexpr size_t SLOT = P0 + 8 * PI;
  static constexpr size_t f_off = 0;
  static constexpr size_t g_off = f_off + RF * SLOT;
  static constexpr size_t phi_off = g_off + RG * SLOT;
  static constexpr size_t bar_off = phi_off + sizeof(T) * TRING * (TBX + 2);
  static constexpr size_t bytes = bar_off + 8 * (RF + RG);
  static_assert(g_off % 16 == 0 && phi_off % 16 == 0 && bar_off % 8 == 0, "smem layout alignment");
  static_assert(P0 % 16 == 0 && PI % 16 == 0, "bulk-copy segments must be 16-byte multiples");
};
// Each try_wait suspends for at most ~1 us (the hint), so a wait gives up
// after about a second; a normal row arrives within microseconds.
constexpr long long MBAR_SPIN_LIMIT = 1LL << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
          smem_u32(bar)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, 1000;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit = MBAR_SPIN_LIMIT) {
  for (long long it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Drain of a block whose bounded wait timed out: wait (with the full bound)
// for the newest phase of every ring slot, i.e. for the copies of the last
// R staged rows [last - R + 1, last] (rows below `first` were never staged).
// An older phase of a slot completed before the slot was staged again, and a
// completed phase returns at once, so only copies still in flight are waited
// for; nothing that was never armed is.  The block's results are invalid
// (the host reports LBM_ECUDA).
__device__ __forceinline__ void drain_ring(uint64_t* bar, int R, int first, int last) {
  for (int r = max(first, last - R + 1); r <= last; ++r) {
    const int li = r - first;
    mbar_wait_bounded(&bar[li % R], (li / R) & 1);
  }
}

// Decoded population i in staged column c of a slot.
template <class C, int SEG>
__device__ __forceinline__ typename C::value_t stg_ld(const unsigned char* slot, int i, int c,
                                                      const typename C::value_t* r2,
                                                      typename C::value_t is) {
  using T = typename C::value_t;
  if constexpr (!C::dev) {
    return reinterpret_cast<const T*>(slot)[i * SEG + c];
  } else {
    const float b = reinterpret_cast<const float*>(slot)[c];
    if (i == 0) return b;
    const uint16_t q = reinterpret_cast<const uint16_t*>(slot + SEG * C::B0)[(i - 1) * SEG + c];
    return fma16(typename C::raw_t(), q, enc16(typename C::raw_t(), is), r2[i >= 5] * b);
  }
}

// Pull of the node in staged column c from the source-row slots rm, r0, rp
// (rows rr-1, rr, rr+1); bounce-back where the source lies beyond a wall.
// r2, is: the set's deviation ratios and inverse scale (PopDev only).
template <class C, int SEG, typename T = typename C::value_t>
__device__ __forceinline__ void pull_staged(const unsigned char* rm, const unsigned char* r0,
                                            const unsigned char* rp, int c, bool bxm, bool bxp, bool bym,
                                            bool byp, const T* r2, T is, T out[9]) {
  out[0] = stg_ld<C, SEG>(r0, 0, c, r2, is);
  out[1] = bxm ? stg_ld<C, SEG>(r0, 3, c, r2, is) : stg_ld<C, SEG>(r0, 1, c - 1, r2, is);
  out[2] = bym ? stg_ld<C, SEG>(r0, 4, c, r2, is) : stg_ld<C, SEG>(rm, 2, c, r2, is);
  out[3] = bxp ? stg_ld<C, SEG>(r0, 1, c, r2, is) : stg_ld<C, SEG>(r0, 3, c + 1, r2, is);
  out[4] = byp ? stg_ld<C, SEG>(r0, 2, c, r2, is) : stg_ld<C, SEG>(rp, 4, c, r2, is);
  out[5] = (bxm || bym) ? stg_ld<C, SEG>(r0, 7, c, r2, is) : stg_ld<C, SEG>(rm, 5, c - 1, r2, is);
  out[6] = (bxp || bym) ? stg_ld<C, SEG>(r0, 8, c, r2, is) : stg_ld<C, SEG>(rm, 6, c + 1, r2, is);
  out[7] = (bxp || byp) ? stg_ld<C, SEG>(r0, 5, c, r2, is) : stg_ld<C, SEG>(rp, 7, c + 1, r2, is);
  out[8] = (bxm || byp) ? stg_ld<C, SEG>(r0, 6, c, r2, is) : stg_ld<C, SEG>(rp, 8, c - 1, r2, is);
}

// The same pull where the reflecting links come from a node's link word m
// (P.obs: bit i-1 set when link i's upstream node is solid or beyond a wall).
template <class C, int SEG, typename T = typename C::value_t>
__device__ __forceinline__ void pull_staged_obs(const unsigned char* rm, const unsigned char* r0,
                                                const unsigned char* rp, int c, unsigned m, const T* r2, T is,
                                                T out[9]) {
  out[0] = stg_ld<C, SEG>(r0, 0, c, r2, is);
  out[1] = (m & 1u) ? stg_ld<C, SEG>(r0, 3, c, r2, is) : stg_ld<C, SEG>(r0, 1, c - 1, r2, is);
  out[2] = (m & 2u) ? stg_ld<C, SEG>(r0, 4, c, r2, is) : stg_ld<C, SEG>(rm, 2, c, r2, is);
  out[3] = (m & 4u) ? stg_ld<C, SEG>(r0, 1, c, r2, is) : stg_ld<C, SEG>(r0, 3, c + 1, r2, is);
  out[4] = (m & 8u) ? stg_ld<C, SEG>(r0, 2, c, r2, is) : stg_ld<C, SEG>(rp, 4, c, r2, is);
  out[5] = (m & 16u) ? stg_ld<C, SEG>(r0, 7, c, r2, is) : stg_ld<C, SEG>(rm, 5, c - 1, r2, is);
  out[6] = (m & 32u) ? stg_ld<C, SEG>(r0, 8, c, r2, is) : stg_ld<C, SEG>(rm, 6, c + 1, r2, is);
  out[7] = (m & 64u) ? stg_ld<C, SEG>(r0, 5, c, r2, is) : stg_ld<C, SEG>(rp, 7, c + 1, r2, is);
  out[8] = (m & 128u) ? stg_ld<C, SEG>(r0, 6, c, r2, is) : stg_ld<C, SEG>(rp, 8, c - 1, r2, is);
}

// Launch shape of the TMA step per storage codec: strip width, rows staged
// ahead of need (f, g), resident threads per SM it is compiled for
// (registers), and whether the f pulled for phi of row y+1 is kept in
// registers for that row's collision instead of being pulled again.
//   FP32: 160 columns, f one row ahead, g two, 4 blocks (20 warps) per SM:
//         shared memory (56 KB a block) is the occupancy limit.  f is kept
//         from phi's pass (SLIM), and the f slot that frees holds the extra g
//         row.
//   FP64: 160 columns, one row ahead, one block per SM (registers).
//   16-bit deviations: 128 columns, two rows ahead, 6 blocks (24 warps) per
//         SM; the rows are 44 % smaller, so more blocks fit, and keeping f
//         saves the second decode.
// Measured on the 16384^2 step (GLUPS): FP32 160/1/1 29.5-30.6 against 128
// to 256 columns, deeper staging or more blocks 24.9-28.2.  FP16 deviations
// 128/2/2 x6 with kept f 34.4; 160/1/1 x4 30.3; 160/2/2 x5 32.3, with kept
// f 33.4; 96/2/2 x8 33.1; 256/2/2 x3 32.5; history staged by TMA or copies
// issued from every warp 27-29.  Keeping f in FP32 too, which frees the f
// ring's row y-1 and lets f be staged two rows ahead in the same shared
// memory (the segment's first phi row then pulled from global memory):
// FP32 30.6 (unchanged), FP16 deviations 32.3 (register spills); the same
// ring with g staged two rows ahead instead: FP32 32.0.  Without the per-row
// block barrier (each warp keeping its own phi ring and re-forming its halo
// columns, row slots recycled through per-slot mbarriers that every warp
// arrives on): FP32 29.2, FP16 deviations 27.2, so the barrier stays.
// FP16 deviations with the f ring starting at row y0-1 as in FP32 and 7
// blocks (28 warps) per SM: 33.9 against 34.8 (46 B of spills at 72
// registers).
template <class C>
struct TmaCfg {
  static constexpr int TBX = C::dev ? 128 : 160;
  static constexpr bool fp32 = !C::dev && sizeof(typename C::value_t) == 4;
  static constexpr int DF = C::dev ? 2 : 1, DG = (C::dev || fp32) ? 2 : 1;
  static constexpr int threads = C::dev ? 768 : (sizeof(typename C::value_t) == 4 ? 640 : 256);
  static constexpr bool keep_f = C::dev || fp32;
  static constexpr bool slim = fp32;
};

// VSEG: segments of P.seg_rows rows (small grids) instead of the constant LY.
// OBS: solid obstacles (P.obs).  phi, with the neutral-wetting values at
// solid nodes, comes from the plane B.phis (written by k_obs_phi and
// k_obs_fill before the launch) instead of from the staged rows; the pulls
// reflect the links flagged in each node's link word; solid nodes store
// zeros.  The staging, rings and barriers are those of the plain step.
template <class C, bool UR, bool VSEG = false, bool OBS = false>
__global__ void __launch_bounds__(TmaCfg<C>::TBX, TmaCfg<C>::threads / TmaCfg<C>::TBX)
    k_step_tma(const Phys<typename C::value_t> P, const Bufs<typename C::value_t> B, int* __restrict__ err) {
  using T = typename C::value_t;
  constexpr int TBX = TmaCfg<C>::TBX, DF = TmaCfg<C>::DF, DG = TmaCfg<C>::DG;
  constexpr bool FK = TmaCfg<C>::keep_f;
  constexpr bool SLIM = TmaCfg<C>::slim;  // (implies FK) the f ring starts at row y0 - 1
  using L = TmaLayout<C, TBX, DF, DG, SLIM>;
  constexpr int SEG = L::SEG, RF = L::RF, RG = L::RG;
  constexpr int FS = (int)L::SLOT;  // bytes per row slot
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* const sf = smem + L::f_off;              // [RF] row slots
  unsigned char* const sg = smem + L::g_off;              // [RG] row slots
  T* const sp = reinterpret_cast<T*>(smem + L::phi_off);  // [TRING][TBX + 2]
  uint64_t* const barF = reinterpret_cast<uint64_t*>(smem + L::bar_off);
  uint64_t* const barG = barF + RF;

  const int tid = threadIdx.x;
  const int nx = P.nx, ny = P.ny;
  const int seg = VSEG ? P.seg_rows : LY;
  const int x0 = blockIdx.x * TBX, y0 = blockIdx.y * seg;
  const int w = min(TBX, nx - x0);
  const int y1 = min(y0 + seg, ny);
  const bool active = tid < w;
  const int x = x0 + tid;
  const bool wx = P.wall_x != 0, wy = P.wall_y != 0;
  const int fbase = y0 - (SLIM ? 1 : 2), gbase = y0 - 1;  // first staged f / g row
  // bytes copied per plane segment: [x0 - XPAD, x0 + w + XPAD) rounded up to 16
  const uint32_t seg0 = (uint32_t)((((w + 2 * XPAD) * C::B0 + 15) / 16) * 16);
  const uint32_t segI = (uint32_t)((((w + 2 * XPAD) * C::BI + 15) / 16) * 16);
  const long long RB = pop_row_bytes<C>(P.pitch);
  // deviation constants of the two sets (unused by PopPlain)
  const T rf2[2] = {P.dv_r[0][0], P.dv_r[0][1]}, rg2[2] = {P.dv_r[1][0], P.dv_r[1][1]};
  const T isf = P.dv_is[0], isg = P.dv_is[1];
  const int f_last = y1 + 1, g_last = y1;  // last f / g row any output row needs
  const bool edge_x = wx && (x0 == 0 || x0 + w == nx);  // strip touches an x wall
  // OBS: this block reaches a solid node (else it runs the plain step's path)
  const bool near = OBS && (!P.obs_near || P.obs_near[blockIdx.y * gridDim.x + blockIdx.x]);

  if (tid == 0) {
    for (int k = 0; k < RF + RG; ++k) mbar_init(&barF[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Launched as a programmatic dependent of the kernel before it on the
  // stream: the next kernel may be scheduled once every block of this one
  // has started, and (without obstacles) every block waits for the kernel
  // before it to finish before any global access.  With obstacles that
  // kernel is the phi pass, which the blocks far from the obstacle do not
  // read; the near blocks wait below.
  asm volatile("griddepcontrol.launch_dependents;");
  if (!OBS) asm volatile("griddepcontrol.wait;" ::: "memory");

  auto wrap_row = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };
  // producer side (thread 0 only)
  auto stage = [&](const void* src, unsigned char* slot, uint64_t* bar, int r) {
    if ((r < 0 || r >= ny) && wy) {  // beyond a wall: nothing to load, complete the phase
      mbar_arrive(bar);
      return;
    }
    // element x0 - XPAD of the row's planes
    const unsigned char* row = static_cast<const unsigned char*>(src) + (long long)wrap_row(r) * RB;
    mbar_arrive_expect_tx(bar, seg0 + 8u * segI);
    bulk_g2s(slot, row + (long long)x0 * C::B0, seg0, bar);
#pragma unroll 1
    for (int i = 1; i < 9; ++i)
      bulk_g2s(slot + L::P0 + (i - 1) * L::PI, row + pop_plane_off<C>(P.pitch, i) + (long long)x0 * C::BI,
               segI, bar);
  };
  // the same issued by lanes 0..8 of warp 0, one plane each (every lane of
  // warp 0 calls it; tid is the lane there)
  auto stage_lanes = [&](const void* src, unsigned char* slot, uint64_t* bar, int r) {
    if ((r < 0 || r >= ny) && wy) {
      if (tid == 0) mbar_arrive(bar);
      return;
    }
    const unsigned char* row = static_cast<const unsigned char*>(src) + (long long)wrap_row(r) * RB;
    if (tid == 0) mbar_arrive_expect_tx(bar, seg0 + 8u * segI);
    if (tid < 9)
      bulk_g2s(slot + (tid ? L::P0 + (tid - 1) * L::PI : 0),
               row + pop_plane_off<C>(P.pitch, tid) + (long long)x0 * (tid ? C::BI : C::B0), tid ? segI : seg0, bar);
  };
  auto fslot = [&](int r) { return sf + ((r - fbase) % RF) * FS; };
  auto gslot = [&](int r) { return sg + ((r - gbase) % RG) * FS; };
  auto wait_f = [&](int r) {
    const int li = r - fbase;
    return mbar_wait_bounded(&barF[li % RF], (li / RF) & 1);
  };
  auto wait_g = [&](int r) {
    const int li = r - gbase;
    return mbar_wait_bounded(&barG[li % RG], (li / RG) & 1);
  };

  // phi of row r (in the domain, or wrapped) into the phi ring: own column,
  // left halo (thread 0), right halo (thread w - 1); x-wall ghosts from the
  // thread's own phi and a second pull of the neighbouring column.
  T fnext[9];  // FK: the pulled f of the last phi row made with keep set
  unsigned mnext = 0;  // OBS and FK: the link word of that row's node
  // OBS: phi of row r from the filled plane (x-wall ghosts as in the plain
  // step, from the plane's columns 0, 1 and nx-1, nx-2).  The plane values
  // and the link word (FK) of a row are loaded one march step before the
  // row is formed, so that their latency overlaps a node update.
  int pre_r = INT_MIN;  // the row whose values the pre_ registers hold
  T pre_c = T(0), pre_l0 = T(0), pre_l1 = T(0), pre_r0 = T(0), pre_r1 = T(0);
  unsigned pre_m = 0;
  const bool wl = wx && x0 == 0, wr = wx && x0 + w == nx;  // the strip ends at an x wall
  auto plane_load = [&](int r) {
    pre_r = r;
    if (!active) return;
    const int rr = wrap_row(r);
    const T* pr = B.phis + ix(P, 1, 0, 0, rr);
    pre_c = pr[x];
    if (FK) pre_m = P.obs[(long long)rr * nx + x];
    if (tid == 0) {
      pre_l0 = x0 > 0 ? pr[x0 - 1] : (!wx ? pr[nx - 1] : pr[0]);
      if (wl) pre_l1 = pr[1];
    }
    if (tid == w - 1) {
      pre_r0 = x0 + w < nx ? pr[x0 + w] : (!wx ? pr[0] : pr[nx - 1]);
      if (wr) pre_r1 = pr[nx - 2];
    }
  };
  // returns the link word of row r's node (FK)
  auto phi_row_plane = [&](int r) -> unsigned {
    if (pre_r != r) plane_load(r);
    T* dst = sp + tslot(r) * (TBX + 2);
    const unsigned m = pre_m;
    if (active) {
      dst[tid + 1] = pre_c;
      if (tid == 0) dst[0] = wl ? wall_ghost(P, SIDE_LEFT, pre_l0, pre_l1) : pre_l0;
      if (tid == w - 1) dst[w + 1] = wr ? wall_ghost(P, SIDE_RIGHT, pre_r0, pre_r1) : pre_r0;
    }
    if (r + 1 <= y1 && (r + 1 < ny || !wy)) plane_load(r + 1);  // the next phi row of the march
    return m;
  };
  auto phi_row_at = [&](int r, const unsigned char* rm, const unsigned char* r0, const unsigned char* rp,
                        bool keep) {
    const int rr = wrap_row(r);
    const bool bym = wy && rr == 0, byp = wy && rr == ny - 1;
    T* dst = sp + tslot(r) * (TBX + 2);
    if (OBS && near) {
      const unsigned m = phi_row_plane(r);
      if (FK && keep && active) {
        mnext = m;
        pull_staged_obs<C, SEG>(rm, r0, rp, tid + XPAD, mnext, rf2, isf, fnext);
      }
      return;
    }
    if (!active) return;
    T v[9];
    if (edge_x || bym || byp)
      pull_staged<C, SEG>(rm, r0, rp, tid + XPAD, wx && x == 0, wx && x == nx - 1, bym, byp, rf2, isf, v);
    else
      pull_staged<C, SEG>(rm, r0, rp, tid + XPAD, false, false, false, false, rf2, isf, v);
    const T ph = sum9(v);
    dst[tid + 1] = ph;
    if (FK && keep) {
#pragma unroll
      for (int i = 0; i < 9; ++i) fnext[i] = v[i];
    }
    if (tid == 0) {
      T hv;
      if (x0 > 0 || !wx) {
        pull_staged<C, SEG>(rm, r0, rp, XPAD - 1, false, wx && x0 - 1 == nx - 1, bym, byp, rf2, isf, v);
        hv = sum9(v);
      } else {
        pull_staged<C, SEG>(rm, r0, rp, XPAD + 1, false, wx && 1 == nx - 1, bym, byp, rf2, isf, v);
        hv = wall_ghost(P, SIDE_LEFT, ph, sum9(v));
      }
      dst[0] = hv;
    }
    if (tid == w - 1) {
      T hv;
      if (x0 + w < nx || !wx) {
        pull_staged<C, SEG>(rm, r0, rp, XPAD + w, wx && x0 + w == 0, wx && x0 + w == nx - 1, bym, byp, rf2, isf, v);
        hv = sum9(v);
      } else {
        pull_staged<C, SEG>(rm, r0, rp, XPAD + w - 2, wx && nx - 2 == 0, false, bym, byp, rf2, isf, v);
        hv = wall_ghost(P, SIDE_RIGHT, ph, sum9(v));
      }
      dst[w + 1] = hv;
    }
  };
  auto phi_row = [&](int r) { phi_row_at(r, fslot(r - 1), fslot(r), fslot(r + 1), r == y0); };
  // SLIM: phi of row y0 - 1 (in the domain or wrapped) from pulls of the
  // global planes, since its f rows are not staged.
  auto phi_row_global = [&](int r) {
    if (OBS && near) {
      phi_row_plane(r);
      return;
    }
    const int rr = wrap_row(r);
    T* dst = sp + tslot(r) * (TBX + 2);
    if (!active) return;
    const T ph = phi_at<C, MODE_STEP>(P, B, x, rr);
    dst[tid + 1] = ph;
    if (tid == 0) {
      T hv;
      if (x0 > 0) hv = phi_at<C, MODE_STEP>(P, B, x0 - 1, rr);
      else if (!wx) hv = phi_at<C, MODE_STEP>(P, B, nx - 1, rr);
      else hv = wall_ghost(P, SIDE_LEFT, ph, phi_at<C, MODE_STEP>(P, B, 1, rr));
      dst[0] = hv;
    }
    if (tid == w - 1) {
      T hv;
      if (x0 + w < nx) hv = phi_at<C, MODE_STEP>(P, B, x0 + w, rr);
      else if (!wx) hv = phi_at<C, MODE_STEP>(P, B, 0, rr);
      else hv = wall_ghost(P, SIDE_RIGHT, ph, phi_at<C, MODE_STEP>(P, B, nx - 2, rr));
      dst[w + 1] = hv;
    }
  };
  auto ghost_row = [&](int rg, int r1, int r2, int side) {
    T* d = sp + tslot(rg) * (TBX + 2);
    const T* a = sp + tslot(r1) * (TBX + 2);
    const T* b = sp + tslot(r2) * (TBX + 2);
    for (int j = tid; j < w + 2; j += TBX) d[j] = wall_ghost(P, side, a[j], b[j]);
  };

  bool ok = true;
  // ---------------------------------------------------------------- prologue
  // f rows fbase .. y0+1+DF and g rows y0-1 .. y0+DG in flight; phi of rows
  // y0-1 and y0 (and of row 1 when the segment starts at a bottom wall, so
  // that the ghost row below it can be formed before the march).
  const bool bottom = wy && y0 == 0;
  if (tid == 0) {
    for (int r = fbase; r <= min(y0 + 1 + DF, f_last); ++r) stage(B.fin, fslot(r), &barF[(r - fbase) % RF], r);
    for (int r = gbase; r <= min(y0 + DG, g_last); ++r) stage(B.gin, gslot(r), &barG[(r - gbase) % RG], r);
  }
  // OBS: the phi plane comes from the pass launched before this kernel,
  // which may still be running (this kernel is its programmatic dependent)
  if (OBS && near) asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int r = fbase; r <= min(y0 + (bottom ? 2 : 1), f_last); ++r) ok = wait_f(r) && ok;
  for (int r = gbase; r <= min(y0, g_last); ++r) ok = wait_g(r) && ok;
  for (int r = y0 - 1; r <= y0 + (bottom ? 1 : 0); ++r) {
    if ((r >= 0 && r < ny) || !wy) {
      if (SLIM && r == y0 - 1) phi_row_global(r);
      else phi_row(r);
    }
  }
  bool failed = __syncthreads_or(!ok);
  if (!failed && bottom) {
    ghost_row(-1, 0, 1, SIDE_BOTTOM);
    __syncthreads();
  }
  T h[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (active) {
    const T* hb = B.hist + ix(P, 5, 0, x, y0);
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k] = hb[k * P.pitch];
  }

  // ---------------------------------------------------------------- march
  // Ring positions advance by one slot per row: f slot of row y and g slot
  // of row y-1, and slot + phase parity of the rows waited for (f row y+2,
  // g row y+1), kept as counters instead of modulo arithmetic.
  auto next = [](int s, int R) { return s + 1 == R ? 0 : s + 1; };
  auto add = [](int s, int k, int R) { return s + k >= R ? s + k - R : s + k; };
  constexpr int LF0 = SLIM ? 1 : 2;                        // local index of f row y0
  int fR0 = LF0 % RF, gA = 0;                              // f row y0, g row y0-1
  int fW = (LF0 + 2) % RF, fWp = ((LF0 + 2) / RF) & 1;     // f row y0+2
  int gW = 2 % RG, gWp = (2 / RG) & 1;       // g row y0+1 (local 2)
  int y = y0;  // on failure: the march step that stopped (rows above it staged by the step before)
  for (; y < y1 && !failed; ++y) {
    ok = true;
    if (y + 2 <= f_last) ok = mbar_wait_bounded(&barF[fW], fWp) && ok;
    if (y + 1 <= g_last) ok = mbar_wait_bounded(&barG[gW], gWp) && ok;
    T f[9];  // pulled f of row y (FK: made with phi of row y)
    unsigned mc = 0;  // OBS: link word of the node of row y
    if (FK) {
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = fnext[i];
      mc = mnext;
    }
    const unsigned char* f_m = sf + add(fR0, RF - 1, RF) * FS;  // f row y-1 (not SLIM)
    const unsigned char* f_0 = sf + fR0 * FS;                   // f row y
    const unsigned char* f_p = sf + add(fR0, 1, RF) * FS;       // f row y+1
    // phi of row y+1 (a ghost row above a top wall)
    const int r1 = y + 1;
    if (r1 < ny || !wy) phi_row_at(r1, f_0, f_p, sf + add(fR0, 2, RF) * FS, true);
    else if (r1 == ny) ghost_row(ny, ny - 1, ny - 2, SIDE_TOP);  // rows ny-1, ny-2 ready since the last barrier
    failed = __syncthreads_or(!ok);
    if (failed) break;
    // the next rows' copies: from lanes 0..8 of warp 0 for FP32 / FP64 sets
    // (+0.7 % for the FP32 step), from thread 0 for the 16-bit codec (the
    // lanes' issue measured 5 % slower there)
    if (C::dev ? tid == 0 : tid < 32) {
      fence_proxy_async_smem();
      if (y + 2 + DF <= f_last) {
        const int sl = add(fR0, 2 + DF, RF);
        if (C::dev) stage(B.fin, sf + sl * FS, &barF[sl], y + 2 + DF);
        else stage_lanes(B.fin, sf + sl * FS, &barF[sl], y + 2 + DF);
      }
      if (y + 1 + DG <= g_last) {
        const int sl = add(gA, 2 + DG, RG);
        if (C::dev) stage(B.gin, sg + sl * FS, &barG[sl], y + 1 + DG);
        else stage_lanes(B.gin, sg + sl * FS, &barG[sl], y + 1 + DG);
      }
    }
    T hn[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (active && y + 1 < y1) {
      const T* hb = B.hist + ix(P, 5, 0, x, y + 1);
#pragma unroll
      for (int k = 0; k < 5; ++k) hn[k] = hb[k * P.pitch];
    }
    if (active) {
      const T* pm = sp + tslot(y - 1) * (TBX + 2);
      const T* p0 = sp + tslot(y) * (TBX + 2);
      const T* pp = sp + tslot(y + 1) * (TBX + 2);
      const int c = tid + 1;
      T phi9[9];
      phi9[0] = p0[c];
      phi9[1] = p0[c + 1];
      phi9[2] = pp[c];
      phi9[3] = p0[c - 1];
      phi9[4] = pm[c];
      phi9[5] = pp[c + 1];
      phi9[6] = pp[c - 1];
      phi9[7] = pm[c - 1];
      phi9[8] = pm[c + 1];
      const unsigned char* g_m = sg + gA * FS;
      const unsigned char* g_0 = sg + add(gA, 1, RG) * FS;
      const unsigned char* g_p = sg + add(gA, 2, RG) * FS;
      const bool bym = wy && y == 0, byp = wy && y == ny - 1;
      T g[9];
      if (OBS && near) {
        if (!FK) mc = P.obs[(long long)y * nx + x];
        if (!FK) pull_staged_obs<C, SEG>(f_m, f_0, f_p, tid + XPAD, mc, rf2, isf, f);
        pull_staged_obs<C, SEG>(g_m, g_0, g_p, tid + XPAD, mc, rg2, isg, g);
      } else if (edge_x || bym || byp) {  // bounce-back links possible (block-uniform test)
        const bool bxm = wx && x == 0, bxp = wx && x == nx - 1;
        if (!FK) pull_staged<C, SEG>(f_m, f_0, f_p, tid + XPAD, bxm, bxp, bym, byp, rf2, isf, f);
        pull_staged<C, SEG>(g_m, g_0, g_p, tid + XPAD, bxm, bxp, bym, byp, rg2, isg, g);
      } else {
        if (!FK) pull_staged<C, SEG>(f_m, f_0, f_p, tid + XPAD, false, false, false, false, rf2, isf, f);
        pull_staged<C, SEG>(g_m, g_0, g_p, tid + XPAD, false, false, false, false, rg2, isg, g);
      }
      if (OBS && near && ((mc >> OBS_SOLID) & 1u)) {  // a solid node: no populations, no history
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = T(0);
        store_pops<C>(P, B.fout, 0, x, y, f, T(0), true);
        store_pops<C>(P, B.gout, 1, x, y, f, T(0), false);
        T* hb = B.hist + ix(P, 5, 0, x, y);
#pragma unroll
        for (int k = 0; k < 5; ++k) hb[k * P.pitch] = T(0);
        if (B.phi_prev) B.phi_prev[ix(P, 1, 0, x, y)] = T(0);
      } else {
        node_update<C, MODEL_AC, MODE_STEP, UR>(P, B, x, y, phi9, phi9, f, g, h, T(0), T(0), T(0));
      }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k] = hn[k];
    fR0 = next(fR0, RF);
    gA = next(gA, RG);
    fW = next(fW, RF);
    if (fW == 0) fWp ^= 1;
    gW = next(gW, RG);
    if (gW == 0) gWp ^= 1;
  }
  if (failed) {
    // record, then let every copy this block issued land (bounded) before
    // the block's shared memory is released; the results of this launch
    // are invalid (the host reports LBM_ECUDA)
    if (tid == 0) {
      atomicOr(err, 1);
      drain_ring(barF, RF, fbase, min(y + 1 + DF, f_last));
      drain_ring(barG, RG, gbase, min(y + DG, g_last));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// TMA-staged fused step, Cahn-Hilliard phase field (D = grad mu_phi, Eq. (6)).
//
// The same staging as k_step_tma, with the wider reach of the CH update: the
// node update of row y reads mu_phi on rows y-1 .. y+1, and mu_phi of a row
// needs the Laplacian of phi (Eq. (5)), so phi runs two rows and two columns
// ahead.  Per march step y: phi of row y+2 from the staged f rows y+1 .. y+3
// (a ghost row above a top wall); block barrier; mu_phi of row y+1 from phi
// rows y .. y+2 (mirrored at walls, as the oracle's ghost rule for mu); the
// node update of row y.  mu_phi is kept per warp: each warp forms it over its
// own 32 columns plus one column on either side (its edge lanes compute the
// outer ones again), so only a warp barrier separates writing it from
// reading it, and a march step has one block barrier.  Segment starts form
// phi of rows y0-2 and y0-1 from pulls of the global planes, and phi of y0,
// y0+1 and mu_phi of y0-1, y0 from the staged rows.
// ---------------------------------------------------------------------------
template <class C>
struct TmaChCfg {
  static constexpr int TBX = 128;
  static constexpr int DF = 1, DG = 1;
  static constexpr int threads = sizeof(typename C::value_t) == 8 ? 256 : 512;
};
constexpr int CH_PRING = 8;  // phi rows (power of two): rows y-2 .. y+2 may be in use
constexpr int CH_MRING = 4;  // mu_phi rows (power of two): rows y-2 .. y+1
constexpr int CH_MWW = 34;   // mu_phi columns of a warp's rows: its 32 and one on either side

template <class C, int TBX, int DF, int DG>
struct TmaChLayout {
  using T = typename C::value_t;
  static constexpr int SEG = Seg<TBX>::value;
  static constexpr int RF = 5 + DF, RG = 3 + DG;  // f rows y-1 .. y+3 live, g rows y-1 .. y+1
  static constexpr int PW = TBX + 4;                // phi columns -2 .. w+1
  static constexpr int MW = ((TBX + 31) / 32) * CH_MWW;  // per warp: mu columns of its lanes, +-1
  static constexpr size_t P0 = (size_t)SEG * C::B0;
  static constexpr size_t PI = (size_t)SEG * C::BI;
  static constexpr size_t SLOT = P0 + 8 * PI;
  static constexpr size_t f_off = 0;
  static constexpr size_t g_off = f_off + RF * SLOT;
  static constexpr size_t phi_off = g_off + RG * SLOT;
  static constexpr size_t mu_off = phi_off + sizeof(T) * CH_PRING * PW;
  static constexpr size_t bar_off = mu_off + sizeof(T) * CH_MRING * MW;
  static constexpr size_t bytes = bar_off + 8 * (RF + RG);
  static_assert(g_off % 16 == 0 && phi_off % 16 == 0 && mu_off % 16 == 0 && bar_off % 8 == 0,
                "smem layout alignment");
  static_assert(P0 % 16 == 0 && PI % 16 == 0, "bulk-copy segments must be 16-byte multiples");
};

// OBS: solid obstacles (P.obs).  In blocks near an obstacle (P.obs_near)
// the phi and mu_phi rows come from the filled planes B.phis and B.mus
// (k_obs_phi, k_obs_mu and k_obs_fill run before the launch over the regions
// those blocks read), with the same wall ghosts and mirrors; the pulls
// reflect the links flagged in each node's link word; solid nodes store
// zeros.  The other blocks run the plain step's path.
template <class C, bool UR, bool VSEG = false, bool OBS = false>
__global__ void __launch_bounds__(TmaChCfg<C>::TBX, TmaChCfg<C>::threads / TmaChCfg<C>::TBX)
    k_step_tma_ch(const Phys<typename C::value_t> P, const Bufs<typename C::value_t> B, int* __restrict__ err) {
  using T = typename C::value_t;
  constexpr int TBX = TmaChCfg<C>::TBX, DF = TmaChCfg<C>::DF, DG = TmaChCfg<C>::DG;
  using L = TmaChLayout<C, TBX, DF, DG>;
  constexpr int SEG = L::SEG, RF = L::RF, RG = L::RG, PW = L::PW, MW = L::MW;
  constexpr int FS = (int)L::SLOT;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* const sf = smem + L::f_off;
  unsigned char* const sg = smem + L::g_off;
  T* const sp = reinterpret_cast<T*>(smem + L::phi_off);  // [CH_PRING][PW], column c at c + 2
  T* const sm = reinterpret_cast<T*>(smem + L::mu_off);   // [CH_MRING][warps][CH_MWW]
  uint64_t* const barF = reinterpret_cast<uint64_t*>(smem + L::bar_off);
  uint64_t* const barG = barF + RF;

  const int tid = threadIdx.x;
  const int nx = P.nx, ny = P.ny;
  const int seg = VSEG ? P.seg_rows : LY;
  const int x0 = blockIdx.x * TBX, y0 = blockIdx.y * seg;
  const int w = min(TBX, nx - x0);
  const int y1 = min(y0 + seg, ny);
  const bool active = tid < w;
  const int x = x0 + tid;
  const bool wx = P.wall_x != 0, wy = P.wall_y != 0;
  const int fbase = y0 - 1, gbase = y0 - 1;  // first staged f / g row
  const uint32_t seg0 = (uint32_t)((((w + 2 * XPAD) * C::B0 + 15) / 16) * 16);
  const uint32_t segI = (uint32_t)((((w + 2 * XPAD) * C::BI + 15) / 16) * 16);
  const long long RB = pop_row_bytes<C>(P.pitch);
  const T rf2[2] = {P.dv_r[0][0], P.dv_r[0][1]}, rg2[2] = {P.dv_r[1][0], P.dv_r[1][1]};
  const T isf = P.dv_is[0], isg = P.dv_is[1];
  const int f_last = y1 + 2, g_last = y1;  // last f / g row any output row needs
  const bool edge_x = wx && (x0 == 0 || x0 + w == nx);
  // OBS: this block reaches a solid node (else it runs the plain step's path)
  const bool near = OBS && (!P.obs_near || P.obs_near[blockIdx.y * gridDim.x + blockIdx.x]);

  if (tid == 0) {
    for (int k = 0; k < RF + RG; ++k) mbar_init(&barF[k], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Launched as a programmatic dependent of the kernel before it on the
  // stream: the next kernel may be scheduled once every block of this one
  // has started, and (without obstacles) every block waits for the kernel
  // before it to finish before any global access.  With obstacles that
  // kernel is the phi pass, which the blocks far from the obstacle do not
  // read; the near blocks wait below.
  asm volatile("griddepcontrol.launch_dependents;");
  if (!OBS) asm volatile("griddepcontrol.wait;" ::: "memory");

  auto wrap_row = [&](int r) { return r < 0 ? r + ny : (r >= ny ? r - ny : r); };
  auto stage = [&](const void* src, unsigned char* slot, uint64_t* bar, int r) {
    if ((r < 0 || r >= ny) && wy) {
      mbar_arrive(bar);
      return;
    }
    const unsigned char* row = static_cast<const unsigned char*>(src) + (long long)wrap_row(r) * RB;
    mbar_arrive_expect_tx(bar, seg0 + 8u * segI);
    bulk_g2s(slot, row + (long long)x0 * C::B0, seg0, bar);
#pragma unroll 1
    for (int i = 1; i < 9; ++i)
      bulk_g2s(slot + L::P0 + (i - 1) * L::PI, row + pop_plane_off<C>(P.pitch, i) + (long long)x0 * C::BI,
               segI, bar);
  };
  // the same issued by lanes 0..8 of warp 0, one plane each (every lane of
  // warp 0 calls it; tid is the lane there)
  auto stage_lanes = [&](const void* src, unsigned char* slot, uint64_t* bar, int r) {
    if ((r < 0 || r >= ny) && wy) {
      if (tid == 0) mbar_arrive(bar);
      return;
    }
    const unsigned char* row = static_cast<const unsigned char*>(src) + (long long)wrap_row(r) * RB;
    if (tid == 0) mbar_arrive_expect_tx(bar, seg0 + 8u * segI);
    if (tid < 9)
      bulk_g2s(slot + (tid ? L::P0 + (tid - 1) * L::PI : 0),
               row + pop_plane_off<C>(P.pitch, tid) + (long long)x0 * (tid ? C::BI : C::B0), tid ? segI : seg0, bar);
  };
  auto fidx = [&](int r) { return (r - fbase) % RF; };
  auto gidx = [&](int r) { return (r - gbase) % RG; };
  auto fslot = [&](int r) { return sf + fidx(r) * FS; };
  auto gslot = [&](int r) { return sg + gidx(r) * FS; };
  auto wait_f = [&](int r) { return mbar_wait_bounded(&barF[fidx(r)], ((r - fbase) / RF) & 1); };
  auto wait_g = [&](int r) { return mbar_wait_bounded(&barG[gidx(r)], ((r - gbase) / RG) & 1); };
  auto prow = [&](int r) { return sp + (r & (CH_PRING - 1)) * PW; };
  const int lane = tid & 31, wbase = tid & ~31;  // this thread's lane, its warp's first column
  // the last active lane of this warp (edge of the strip's last columns)
  const int last_lane = min(31, w - 1 - wbase);
  // mu_phi row r of this warp: column wbase + j at index j + 1 (j = -1 .. 32)
  auto mrow = [&](int r) { return sm + (r & (CH_MRING - 1)) * MW + (tid >> 5) * CH_MWW; };

  // phi of row r (in the domain or wrapped) from the staged slots: own column,
  // thread 0 columns -1 and -2, thread w-1 columns w and w+1; at an x wall the
  // ghost column from the wetting rule (the column beyond it is not needed:
  // mu_phi is mirrored there).
  // OBS: phi of row r from the filled plane, the halo columns as above
  auto phi_row_plane = [&](int r) {
    const int rr = wrap_row(r);
    T* dst = prow(r);
    if (!active) return;
    const T* pr = B.phis + ix(P, 1, 0, 0, rr);
    dst[tid + 2] = pr[x];
    if (tid == 0) {
      if (x0 > 0 || !wx) {
        dst[1] = pr[x0 > 0 ? x0 - 1 : nx - 1];
        dst[0] = pr[x0 > 1 ? x0 - 2 : x0 - 2 + nx];
      } else {
        dst[1] = wall_ghost(P, SIDE_LEFT, pr[0], pr[1]);
        dst[0] = T(0);
      }
    }
    if (tid == w - 1) {
      if (x0 + w < nx || !wx) {
        const int a = x0 + w < nx ? x0 + w : x0 + w - nx;
        const int b = x0 + w + 1 < nx ? x0 + w + 1 : x0 + w + 1 - nx;
        dst[w + 2] = pr[a];
        dst[w + 3] = (wx && x0 + w + 1 == nx) ? wall_ghost(P, SIDE_RIGHT, pr[nx - 1], pr[nx - 2]) : pr[b];
      } else {
        dst[w + 2] = wall_ghost(P, SIDE_RIGHT, pr[nx - 1], pr[nx - 2]);
        dst[w + 3] = T(0);
      }
    }
  };
  // the threads that form the halo columns' phi from staged rows: lane 0 of
  // warps 1 and 2 on strips wider than two warps (thread 0, in warp 0,
  // issues the row copies), threads 0 and w - 1 where a halo column is a
  // wall ghost (it needs their own phi) or the strip is narrower
  const int tl = (w > 64 && !(wx && x0 == 0)) ? 32 : 0;
  const int tr = (w > 64 && !(wx && (x0 + w == nx || x0 + w + 1 == nx))) ? 64 : w - 1;
  auto phi_row_at = [&](int r, const unsigned char* rm, const unsigned char* r0, const unsigned char* rp) {
    if (OBS && near) {
      phi_row_plane(r);
      return;
    }
    const int rr = wrap_row(r);
    const bool bym = wy && rr == 0, byp = wy && rr == ny - 1;
    T* dst = prow(r);
    if (!active) return;
    T v[9];
    if (edge_x || bym || byp)
      pull_staged<C, SEG>(rm, r0, rp, tid + XPAD, wx && x == 0, wx && x == nx - 1, bym, byp, rf2, isf, v);
    else
      pull_staged<C, SEG>(rm, r0, rp, tid + XPAD, false, false, false, false, rf2, isf, v);
    const T ph = sum9(v);
    dst[tid + 2] = ph;
    if (tid == tl) {
      if (x0 > 0 || !wx) {
        pull_staged<C, SEG>(rm, r0, rp, XPAD - 1, false, wx && x0 - 1 == nx - 1, bym, byp, rf2, isf, v);
        dst[1] = sum9(v);
        pull_staged<C, SEG>(rm, r0, rp, XPAD - 2, false, wx && x0 - 2 == nx - 1, bym, byp, rf2, isf, v);
        dst[0] = sum9(v);
      } else {
        pull_staged<C, SEG>(rm, r0, rp, XPAD + 1, false, wx && 1 == nx - 1, bym, byp, rf2, isf, v);
        dst[1] = wall_ghost(P, SIDE_LEFT, ph, sum9(v));
        dst[0] = T(0);
      }
    }
    if (tid == tr) {
      if (x0 + w < nx || !wx) {
        pull_staged<C, SEG>(rm, r0, rp, XPAD + w, wx && x0 + w == 0, wx && x0 + w == nx - 1, bym, byp, rf2, isf,
                            v);
        const T pw = sum9(v);
        dst[w + 2] = pw;
        if (wx && x0 + w + 1 == nx) {  // column w is the last node: w+1 is the wall ghost
          dst[w + 3] = wall_ghost(P, SIDE_RIGHT, pw, ph);
        } else {
          pull_staged<C, SEG>(rm, r0, rp, XPAD + w + 1, false, wx && x0 + w + 1 == nx - 1, bym, byp, rf2, isf, v);
          dst[w + 3] = sum9(v);
        }
      } else {
        pull_staged<C, SEG>(rm, r0, rp, XPAD + w - 2, wx && nx - 2 == 0, false, bym, byp, rf2, isf, v);
        dst[w + 2] = wall_ghost(P, SIDE_RIGHT, ph, sum9(v));
        dst[w + 3] = T(0);
      }
    }
  };
  // the same from pulls of the global planes (segment starts)
  auto phi_row_global = [&](int r) {
    if (OBS && near) {
      phi_row_plane(r);
      return;
    }
    const int rr = wrap_row(r);
    T* dst = prow(r);
    if (!active) return;
    const T ph = phi_at<C, MODE_STEP>(P, B, x, rr);
    dst[tid + 2] = ph;
    if (tid == 0) {
      if (x0 > 0 || !wx) {
        const int a = x0 > 0 ? x0 - 1 : nx - 1, b = x0 > 1 ? x0 - 2 : x0 - 2 + nx;
        dst[1] = phi_at<C, MODE_STEP>(P, B, a, rr);
        dst[0] = phi_at<C, MODE_STEP>(P, B, b, rr);
      } else {
        dst[1] = wall_ghost(P, SIDE_LEFT, ph, phi_at<C, MODE_STEP>(P, B, 1, rr));
        dst[0] = T(0);
      }
    }
    if (tid == w - 1) {
      if (x0 + w < nx || !wx) {
        const int a = x0 + w < nx ? x0 + w : x0 + w - nx;
        const int b = x0 + w + 1 < nx ? x0 + w + 1 : x0 + w + 1 - nx;
        const T pw = phi_at<C, MODE_STEP>(P, B, a, rr);
        dst[w + 2] = pw;
        dst[w + 3] = (wx && x0 + w + 1 == nx) ? wall_ghost(P, SIDE_RIGHT, pw, ph) : phi_at<C, MODE_STEP>(P, B, b, rr);
      } else {
        dst[w + 2] = wall_ghost(P, SIDE_RIGHT, ph, phi_at<C, MODE_STEP>(P, B, nx - 2, rr));
        dst[w + 3] = T(0);
      }
    }
  };
  // ghost phi row beyond a y wall over every ring column, from rows r1, r2
  auto ghost_row = [&](int rg, int r1, int r2, int side) {
    T* d = prow(rg);
    const T* a = prow(r1);
    const T* b = prow(r2);
    for (int j = tid; j < w + 4; j += TBX) d[j] = wall_ghost(P, side, a[j], b[j]);
  };
  // mu_phi (Eq. (5)) at ring column j of a row, from phi rows r-1, r, r+1
  auto mu_at = [&](const T* pm, const T* p0, const T* pp, int j) {
    const T ph = p0[j];
    const T lap = (((p0[j + 1] - ph) + (p0[j - 1] - ph)) + ((pp[j] - ph) + (pm[j] - ph))) * T(2.0 / 3.0) +
                  (((pp[j + 1] - ph) + (pm[j - 1] - ph)) + ((pp[j - 1] - ph) + (pm[j + 1] - ph))) * T(1.0 / 6.0);
    return P.beta4 * (ph - P.phiA) * (ph - P.phiB) * (ph - P.phibar) - P.kappa * lap;
  };
  // mu_phi of row r for this warp: its own columns, and the column beyond
  // either end (lane 0 and the last active lane form those again); at an x
  // wall the column beyond mirrors the column next to the wall
  auto mu_row = [&](int r) {
    const T* pm = prow(r - 1);
    const T* p0 = prow(r);
    const T* pp = prow(r + 1);
    T* d = mrow(r);
    if (!active) return;
    if (OBS && near) {  // from the filled plane, mirrored at x walls
      const T* mr = B.mus + ix(P, 1, 0, 0, wrap_row(r));
      const T mo = mr[x];
      d[lane + 1] = mo;
      if (lane == 0) d[0] = (wx && x == 0) ? mo : mr[x > 0 ? x - 1 : nx - 1];
      if (lane == last_lane) d[lane + 2] = (wx && x == nx - 1) ? mo : mr[x + 1 < nx ? x + 1 : 0];
      return;
    }
    const T mo = mu_at(pm, p0, pp, tid + 2);
    d[lane + 1] = mo;
    if (lane == 0) d[0] = (wx && x == 0) ? mo : mu_at(pm, p0, pp, tid + 1);
    if (lane == last_lane) d[lane + 2] = (wx && x == nx - 1) ? mo : mu_at(pm, p0, pp, tid + 3);
  };
  // mirrored mu_phi row beyond a y wall (this warp's entries)
  auto mu_copy_row = [&](int rdst, int rsrc) {
    T* d = mrow(rdst);
    const T* s = mrow(rsrc);
    for (int j = lane; j < CH_MWW; j += 32) d[j] = s[j];
  };

  bool ok = true;
  // ---------------------------------------------------------------- prologue
  if (tid == 0) {
    for (int r = fbase; r <= min(y0 + 2 + DF, f_last); ++r) stage(B.fin, fslot(r), &barF[fidx(r)], r);
    for (int r = gbase; r <= min(y0 + DG, g_last); ++r) stage(B.gin, gslot(r), &barG[gidx(r)], r);
  }
  // OBS: the planes come from the passes launched before this kernel, the
  // last of which may still be running (this kernel is its programmatic
  // dependent)
  if (OBS && near) asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int r = fbase; r <= min(y0 + 2, f_last); ++r) ok = wait_f(r) && ok;
  for (int r = gbase; r <= min(y0, g_last); ++r) ok = wait_g(r) && ok;
  for (int r = y0 - 2; r <= y0 - 1; ++r)
    if ((r >= 0 && r < ny) || !wy) phi_row_global(r);
  for (int r = y0; r <= y0 + 1; ++r)
    if (r < ny || !wy) phi_row_at(r, fslot(r - 1), fslot(r), fslot(r + 1));
  bool failed = __syncthreads_or(!ok);
  if (!failed && wy && (y0 <= 1 || y0 + 1 == ny)) {
    if (y0 <= 1) ghost_row(-1, 0, 1, SIDE_BOTTOM);
    if (y0 + 1 == ny) ghost_row(ny, ny - 1, ny - 2, SIDE_TOP);
    __syncthreads();
  }
  if (!failed) {
    for (int r = y0 - 1; r <= y0; ++r)
      if ((r >= 0 && r < ny) || !wy) mu_row(r);
    __syncwarp();
    if (wy && y0 == 0) {
      mu_copy_row(-1, 0);
      __syncwarp();
    }
  }
  T h[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (active) {
    const T* hb = B.hist + ix(P, 5, 0, x, y0);
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k] = hb[k * P.pitch];
  }

  // ---------------------------------------------------------------- march
  int y = y0;  // on failure: the march step that stopped (rows above it staged by the step before)
  for (; y < y1 && !failed; ++y) {
    ok = true;
    if (y + 3 <= f_last) ok = wait_f(y + 3) && ok;
    if (y + 1 <= g_last) ok = wait_g(y + 1) && ok;
    const int r2 = y + 2;
    if (r2 < ny || !wy) phi_row_at(r2, fslot(r2 - 1), fslot(r2), fslot(r2 + 1));
    else if (r2 == ny) ghost_row(ny, ny - 1, ny - 2, SIDE_TOP);  // rows ny-1, ny-2 complete
    failed = __syncthreads_or(!ok);
    if (failed) break;
    // the next rows' copies: lanes 0..8 of warp 0 (FP32 / FP64), thread 0
    // (16-bit codec), as in the Allen-Cahn step
    if (C::dev ? tid == 0 : tid < 32) {
      fence_proxy_async_smem();
      const int rf = y + 3 + DF, rg = y + 1 + DG;  // into the slots of rows y-2
      if (C::dev) {
        if (rf <= f_last) stage(B.fin, fslot(rf), &barF[fidx(rf)], rf);
        if (rg <= g_last) stage(B.gin, gslot(rg), &barG[gidx(rg)], rg);
      } else {
        if (rf <= f_last) stage_lanes(B.fin, fslot(rf), &barF[fidx(rf)], rf);
        if (rg <= g_last) stage_lanes(B.gin, gslot(rg), &barG[gidx(rg)], rg);
      }
    }
    const int r1 = y + 1;
    if (r1 < ny || !wy) mu_row(r1);
    else if (r1 == ny) mu_copy_row(ny, ny - 1);
    __syncwarp();
    T hn[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (active && y + 1 < y1) {
      const T* hb = B.hist + ix(P, 5, 0, x, y + 1);
#pragma unroll
      for (int k = 0; k < 5; ++k) hn[k] = hb[k * P.pitch];
    }
    if (active) {
      const T* pm = prow(y - 1);
      const T* p0 = prow(y);
      const T* pp = prow(y + 1);
      const int c = tid + 2;
      T phi9[9];
      phi9[0] = p0[c];
      phi9[1] = p0[c + 1];
      phi9[2] = pp[c];
      phi9[3] = p0[c - 1];
      phi9[4] = pm[c];
      phi9[5] = pp[c + 1];
      phi9[6] = pp[c - 1];
      phi9[7] = pm[c - 1];
      phi9[8] = pm[c + 1];
      const T* mm = mrow(y - 1);
      const T* m0 = mrow(y);
      const T* mp = mrow(y + 1);
      const int cm = lane + 1;
      T mu9[9];
      mu9[0] = m0[cm];
      mu9[1] = m0[cm + 1];
      mu9[2] = mp[cm];
      mu9[3] = m0[cm - 1];
      mu9[4] = mm[cm];
      mu9[5] = mp[cm + 1];
      mu9[6] = mp[cm - 1];
      mu9[7] = mm[cm - 1];
      mu9[8] = mm[cm + 1];
      const bool bym = wy && y == 0, byp = wy && y == ny - 1;
      T f[9], g[9];
      unsigned mc = 0;
      if (OBS && near) {
        mc = P.obs[(long long)y * nx + x];
        pull_staged_obs<C, SEG>(fslot(y - 1), fslot(y), fslot(y + 1), tid + XPAD, mc, rf2, isf, f);
        pull_staged_obs<C, SEG>(gslot(y - 1), gslot(y), gslot(y + 1), tid + XPAD, mc, rg2, isg, g);
      } else if (edge_x || bym || byp) {
        const bool bxm = wx && x == 0, bxp = wx && x == nx - 1;
        pull_staged<C, SEG>(fslot(y - 1), fslot(y), fslot(y + 1), tid + XPAD, bxm, bxp, bym, byp, rf2, isf, f);
        pull_staged<C, SEG>(gslot(y - 1), gslot(y), gslot(y + 1), tid + XPAD, bxm, bxp, bym, byp, rg2, isg, g);
      } else {
        pull_staged<C, SEG>(fslot(y - 1), fslot(y), fslot(y + 1), tid + XPAD, false, false, false, false, rf2,
                            isf, f);
        pull_staged<C, SEG>(gslot(y - 1), gslot(y), gslot(y + 1), tid + XPAD, false, false, false, false, rg2,
                            isg, g);
      }
      if (OBS && near && ((mc >> OBS_SOLID) & 1u)) {  // a solid node: no populations, no history
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = T(0);
        store_pops<C>(P, B.fout, 0, x, y, f, T(0), true);
        store_pops<C>(P, B.gout, 1, x, y, f, T(0), false);
        T* hb = B.hist + ix(P, 5, 0, x, y);
#pragma unroll
        for (int k = 0; k < 5; ++k) hb[k * P.pitch] = T(0);
        if (B.phi_prev) B.phi_prev[ix(P, 1, 0, x, y)] = T(0);
      } else {
        node_update<C, MODEL_CH, MODE_STEP, UR>(P, B, x, y, phi9, mu9, f, g, h, T(0), T(0), T(0));
      }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) h[k] = hn[k];
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(err, 1);
      drain_ring(barF, RF, fbase, min(y + 2 + DF, f_last));
      drain_ring(barG, RG, gbase, min(y + DG, g_last));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Auxiliary kernels: gather the pulled populations, scatter populations back
// into the pre-stream layout, convert planes, diagnostics reductions.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_pull(const Phys<T> P, const T* __restrict__ in, T* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  T v[9];
  if (P.obs)
    pull9_obs<PopPlain<T>>(in, P, 0, x, y, v);
  else
    pull9<PopPlain<T>>(in, P, 0, x, y, v);
  T* o = out + ix(P, 9, 0, x, y);
#pragma unroll
  for (int i = 0; i < 9; ++i) o[i * P.pitch] = v[i];
}

// Inverse of the pull: the population node x sees in direction i came from
// x - c_i (or, beyond a wall or from a solid node, from x itself in
// direction opp(i)).  Every destination entry a fluid node pulls is written
// exactly once; solid nodes scatter nothing (no fluid node reads them).
template <typename T>
__global__ void k_unstream(const Phys<T> P, const T* __restrict__ in, T* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  const unsigned m = P.obs ? P.obs[(long long)y * P.nx + x] : 0u;
  if ((m >> OBS_SOLID) & 1u) return;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    int sx = x - cx[i], sy = y - cy[i];
    bool wall = i > 0 && ((m >> (i - 1)) & 1u);
    if (sx < 0 || sx >= P.nx) { if (P.wall_x) wall = true; else sx = (sx + P.nx) % P.nx; }
    if (sy < 0 || sy >= P.ny) { if (P.wall_y) wall = true; else sy = (sy + P.ny) % P.ny; }
    const T val = in[ix(P, 9, i, x, y)];
    const int dx = wall ? x : sx, dy = wall ? y : sy, di = wall ? op[i] : i;
    const long long d = ix(P, 9, di, dx, dy);
    out[d] = val;
    if (!P.wall_x) {  // periodic copies in the row pads
      if (dx < XPAD) out[d + P.nx] = val;
      if (dx >= P.nx - XPAD) out[d - P.nx] = val;
    }
  }
}

// Deviation storage: the pulled population k of the nodes of the region
// [x0, x0+w) x [y0, y0+hgt), decoded, as dense doubles plus add.
template <class C>
__global__ void k_pull_export(const Phys<typename C::value_t> P, const void* __restrict__ in, int set, int k,
                              double* __restrict__ out, double add, int x0, int y0, int w, int hgt) {
  using T = typename C::value_t;
  const int xx = blockIdx.x * blockDim.x + threadIdx.x;
  const int yy = blockIdx.y;
  if (xx >= w) return;
  T v[9];
  if (P.obs) {
    pull9_obs<C>(in, P, set, x0 + xx, y0 + yy, v);
    if ((P.obs[(long long)(y0 + yy) * P.nx + x0 + xx] >> OBS_SOLID) & 1u) add = 0.0;  // solid: zero
  } else {
    pull9<C>(in, P, set, x0 + xx, y0 + yy, v);
  }
  out[(long long)yy * w + xx] = double(v[k]) + add;
}

// Deviation storage: the inverse of the pull, node by node.  Slot j of
// node s receives the value node s + c_j pulls in direction j, or, where
// s + c_j lies beyond a wall or is solid, the value s itself pulls in
// direction opp(j); the node's nine slots are then encoded together (for f
// with the node's zeroth moment kept exact).  Solid nodes store zeros.
template <class C>
__global__ void k_restream(const Phys<typename C::value_t> P, const typename C::value_t* __restrict__ in,
                           void* __restrict__ out, int set) {
  using T = typename C::value_t;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  T v[9];
  const unsigned m = P.obs ? P.obs[(long long)y * P.nx + x] : 0u;
  if ((m >> OBS_SOLID) & 1u) {
#pragma unroll
    for (int j = 0; j < 9; ++j) v[j] = T(0);
    store_pops<C>(P, out, set, x, y, v, T(0), set == 0);
    return;
  }
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int tx = x + cx[j], ty = y + cy[j];
    // link opp(j) of s starts at s + c_j
    bool wall = j > 0 && ((m >> (op[j] - 1)) & 1u);
    if (tx < 0 || tx >= P.nx) { if (P.wall_x) wall = true; else tx = (tx + P.nx) % P.nx; }
    if (ty < 0 || ty >= P.ny) { if (P.wall_y) wall = true; else ty = (ty + P.ny) % P.ny; }
    v[j] = wall ? in[ix(P, 9, op[j], x, y)] : in[ix(P, 9, j, tx, ty)];
  }
  store_pops<C>(P, out, set, x, y, v, sum9(v), set == 0);
}

// plane k of a set of NP interleaved planes -> dense doubles of the region
// [x0, x0+w) x [y0, y0+hgt), plus add (not at solid nodes, which export zero)
template <typename T>
__global__ void k_export(const Phys<T> P, const T* __restrict__ in, int NP, int k, double* __restrict__ out,
                         double add, int x0, int y0, int w, int hgt) {
  const int xx = blockIdx.x * blockDim.x + threadIdx.x;
  const int yy = blockIdx.y;
  if (xx >= w) return;
  if (P.obs && ((P.obs[(long long)(y0 + yy) * P.nx + x0 + xx] >> OBS_SOLID) & 1u)) add = 0.0;
  out[(long long)yy * w + xx] = double(in[ix(P, NP, k, x0 + xx, y0 + yy)]) + add;
}

// dense doubles (one plane) minus sub -> plane k of a set of NP interleaved planes
template <typename T>
__global__ void k_import(const Phys<T> P, const double* __restrict__ in, T* __restrict__ out, int NP, int k,
                         double sub) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  out[ix(P, NP, k, x, y)] = T(in[(long long)y * P.nx + x] - sub);
}

// Diagnostics, Eqs. (42)-(43), from the MACRO planes and phi(t-1).
// Per block: [sum phi, sum trS^2, sum S_m^2, max|u|, non-finite, count].
// Sums and maxima run over the fluid nodes; the averages skip nodes next to
// a wall or a solid node (a reflecting link).
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_FIELDS = 6;

__device__ __forceinline__ void warp_reduce6(double v[DIAG_FIELDS]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < DIAG_FIELDS; ++k) {
      const double other = __shfl_down_sync(0xffffffffu, v[k], o);
      v[k] = (k == 3) ? fmax(v[k], other) : v[k] + other;
    }
  }
}

__device__ __forceinline__ void block_reduce6(double v[DIAG_FIELDS], double* out) {
  __shared__ double red[DIAG_THREADS / 32][DIAG_FIELDS];
  warp_reduce6(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < DIAG_FIELDS; ++k) red[wid][k] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < DIAG_FIELDS; ++k)
      v[k] = lane < DIAG_THREADS / 32 ? red[lane][k] : 0.0;
    warp_reduce6(v);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < DIAG_FIELDS; ++k) out[k] = v[k];
  }
}

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_partial(const Phys<T> P, const T* __restrict__ mac,
                                                               const T* __restrict__ phi_prev,
                                                               double* __restrict__ partial) {
  double v[DIAG_FIELDS] = {0, 0, 0, 0, 0, 0};
  const long long N = (long long)P.nx * P.diag_y1;
  const long long pl = P.pitch;  // macro plane k of a node sits k * pitch after plane 0
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const double wi[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  for (long long n = (long long)P.nx * P.diag_y0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
       n += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(n / P.nx), x = (int)(n - (long long)y * P.nx);
    const unsigned om = P.obs ? P.obs[n] : 0u;
    if ((om >> OBS_SOLID) & 1u) continue;
    const long long id = ix(P, NMACRO, 0, x, y);
    const double phi = double(mac[MAC_PHI * pl + id]);
    const double u = double(mac[MAC_UX * pl + id]), vv = double(mac[MAC_UY * pl + id]);
    const double um2 = u * u + vv * vv;
    v[0] += phi;
    if (!isfinite(phi) || !isfinite(um2)) {
      v[4] += 1.0;
    } else {
      v[3] = fmax(v[3], sqrt(um2));
    }
    if ((P.wall_x && (x == 0 || x == P.nx - 1)) || (P.wall_y && (y == 0 || y == P.ny - 1))) continue;
    if (om & 0xffu) continue;
    const double trS = double(mac[MAC_TRS * pl + id]);
    double div = 0.0;
#pragma unroll
    for (int k = 1; k < 9; ++k) {
      int xn = x + cx[k], yn = y + cy[k];
      xn = xn < 0 ? xn + P.nx : (xn >= P.nx ? xn - P.nx : xn);
      yn = yn < 0 ? yn + P.ny : (yn >= P.ny ? yn - P.ny : yn);
      const long long q = ix(P, NMACRO, 0, xn, yn);
      const double rq = double(mac[MAC_RHO * pl + q]);
      const double Jx = rq * double(mac[MAC_UX * pl + q]) + double(mac[MAC_MCX * pl + q]);
      const double Jy = rq * double(mac[MAC_UY * pl + q]) + double(mac[MAC_MCY * pl + q]);
      div += wi[k] * (cx[k] * Jx + cy[k] * Jy) * 3.0;
    }
    const double sm = double(P.drho) * (phi - double(phi_prev[ix(P, 1, 0, x, y)])) + div;
    v[1] += trS * trS;
    v[2] += sm * sm;
    v[5] += 1.0;
  }
  block_reduce6(v, partial + (long long)blockIdx.x * DIAG_FIELDS);
}

template <typename T>
__global__ void __launch_bounds__(DIAG_THREADS) k_diag_final(const double* __restrict__ partial,
                                                             int nparts, double* __restrict__ out) {
  double v[DIAG_FIELDS] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
#pragma unroll
    for (int k = 0; k < DIAG_FIELDS; ++k)
      v[k] = (k == 3) ? fmax(v[k], partial[b * DIAG_FIELDS + k]) : v[k] + partial[b * DIAG_FIELDS + k];
  }
  block_reduce6(v, out);
}

}  // namespace pflbm
