// Discrete adjoint (reverse mode) of the fused Allen-Cahn step.
//
// The forward step maps the state s_t = (f*, g*, chi) -- post-collision
// populations and the history of the explicit-Euler derivatives -- to
// s_{t+1} (Sec. 3, App. C).  Given lambda_{t+1} = dJ/ds_{t+1}, one adjoint
// step forms lambda_t = (ds_{t+1}/ds_t)^T lambda_{t+1} and adds dJ/dG of the
// step (G = the body-force vector of F = mu_phi grad phi + G), in five
// passes over the grid:
//   k_adj_phi     phi(t) = sum_i f_i of the pulled populations       (Eq. (22a))
//   k_adj_node    per node: the forward node update is recomputed, then
//                 swept in reverse (collisions Eqs. (17), (40); moments of
//                 Eqs. (C.2)-(C.4); p of Eq. (39); u of Eq. (22b); m^{phi C}
//                 of Eq. (15); n, lambda, mu of Eqs. (5), (7)-(8); the
//                 stencils of Eqs. (C.9)-(C.10)).  Out: the adjoint of the nine
//                 phi values of the node's stencil, of its pulled f and g
//                 (through the collisions), of its history input, and its
//                 share of dJ/dG.
//   k_adj_gather  the adjoint of phi on the grid extended by the ghost ring:
//                 each position sums the stencil adjoints that read it.
//   k_adj_fold_y, k_adj_fold_x
//                 the ghost values are functions of the fluid values next to
//                 the wall (Eqs. (49)-(50)); their adjoints are folded back in
//                 the reverse order of construction (y rows, which include the
//                 corners, then x columns).
//   k_adj_stream  the reverse of the pull with half-way bounce-back: the
//                 adjoint of f*_j(s) is that of the pulled f_j(s + c_j) plus
//                 phi's adjoint there (phi = sum of the pulled f), or of
//                 f_opp(j)(s) where s + c_j lies beyond a wall.
// The step is smooth (n = grad phi / (|grad phi|^4 + delta_n^4)^(1/4)) except
// for the wetting root's clamped discriminant, whose derivative is taken as
// zero where the clamp acts.
#pragma once

#include "pflbm_kernels.cuh"

namespace pflbm {

constexpr int ADJ_THREADS = 128;

// phi at an extended position (x in [-1, nx], y in [-1, ny]) of the plane
// phi: x sides first (wrap or wetting ghost), then y sides over the extended
// x range -- the construction the forward kernels use.
template <typename T>
__device__ __forceinline__ T phi_xext(const Phys<T>& P, const T* phi, int x, int y) {
  if (x < 0 || x >= P.nx) {
    if (!P.wall_x) return phi[ix(P, 1, 0, x < 0 ? x + P.nx : x - P.nx, y)];
    if (x < 0) return wall_ghost(P, SIDE_LEFT, phi[ix(P, 1, 0, 0, y)], phi[ix(P, 1, 0, 1, y)]);
    return wall_ghost(P, SIDE_RIGHT, phi[ix(P, 1, 0, P.nx - 1, y)], phi[ix(P, 1, 0, P.nx - 2, y)]);
  }
  return phi[ix(P, 1, 0, x, y)];
}
template <typename T>
__device__ __forceinline__ T phi_ext(const Phys<T>& P, const T* phi, int x, int y) {
  if (y < 0 || y >= P.ny) {
    if (!P.wall_y) return phi_xext(P, phi, x, y < 0 ? y + P.ny : y - P.ny);
    if (y < 0) return wall_ghost(P, SIDE_BOTTOM, phi_xext(P, phi, x, 0), phi_xext(P, phi, x, 1));
    return wall_ghost(P, SIDE_TOP, phi_xext(P, phi, x, P.ny - 1), phi_xext(P, phi, x, P.ny - 2));
  }
  return phi_xext(P, phi, x, y);
}

// Derivatives of the wetting ghost 8/3 phi_w - 2 phi_1 + phi_2 / 3 with
// respect to phi_1 and phi_2, phi_w = 2c / (-b - sqrt(b^2 - 4ac)).
template <typename T>
__device__ __forceinline__ void wall_ghost_d(const Phys<T>& P, int side, T phi1, T phi2, T& d1, T& d2) {
  const T a = P.wa[side];
  const T b = T(8.0 / 3.0) - a * (P.phiA + P.phiB);
  const T c = a * P.phiA * P.phiB + phi2 * T(1.0 / 3.0) - T(3) * phi1;
  const T disc = b * b - T(4) * a * c;
  const bool pos = disc > T(0);
  const T s = pos ? sqrt(disc) : T(0);
  const T Dn = -b - s;
  const T dDn = pos ? T(2) * a / s : T(0);  // d(-b - s)/dc
  const T dw = (T(2) * Dn - T(2) * c * dDn) / (Dn * Dn);  // d phi_w / dc
  d1 = T(8.0 / 3.0) * dw * T(-3) - T(2);
  d2 = T(8.0 / 3.0) * dw * T(1.0 / 3.0) + T(1.0 / 3.0);
}

// out = M v (moments, the basis of Eq. (C.1)) and out = M^T v
template <typename T>
__device__ __forceinline__ void mmul(const T v[9], T m[9]) {
  const T a = (v[1] + v[3]) + (v[2] + v[4]), b = (v[5] + v[7]) + (v[6] + v[8]);
  const T d13 = v[1] - v[3], d24 = v[2] - v[4];
  const T dx = (v[5] - v[7]) + (v[8] - v[6]), dy = (v[5] - v[7]) + (v[6] - v[8]);
  m[0] = v[0] + a + b;
  m[1] = T(-4) * v[0] - a + T(2) * b;
  m[2] = T(4) * v[0] - T(2) * a + b;
  m[3] = d13 + dx;
  m[4] = T(-2) * d13 + dx;
  m[5] = d24 + dy;
  m[6] = T(-2) * d24 + dy;
  m[7] = (v[1] + v[3]) - (v[2] + v[4]);
  m[8] = (v[5] + v[7]) - (v[6] + v[8]);
}
template <typename T>
__device__ __forceinline__ void mtmul(const T v[9], T o[9]) {
  const T r0 = v[0] - v[1] - T(2) * v[2];          // axis directions, common part
  const T r1 = v[0] + T(2) * v[1] + v[2];          // diagonal directions, common part
  const T ax = v[3] - T(2) * v[4], ay = v[5] - T(2) * v[6];
  const T qx = v[3] + v[4], qy = v[5] + v[6];
  o[0] = v[0] - T(4) * v[1] + T(4) * v[2];
  o[1] = r0 + ax + v[7];
  o[2] = r0 + ay - v[7];
  o[3] = r0 - ax + v[7];
  o[4] = r0 - ay - v[7];
  o[5] = r1 + qx + qy + v[8];
  o[6] = r1 - qx + qy - v[8];
  o[7] = r1 - qx - qy + v[8];
  o[8] = r1 + qx - qy - v[8];
}

// Reciprocal squared norms of the rows of M: M^{-1} = M^T diag(1 / |row k|^2).
__device__ __forceinline__ double inv_row_norm2(int k) {
  const double n[9] = {1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 6, 1.0 / 12, 1.0 / 6, 1.0 / 12, 0.25, 0.25};
  return n[k];
}

// ---------------------------------------------------------------------------
// Node adjoint.  In: the node's stencil phi9 (phi at x + c_k), pulled f, g,
// history h, and the adjoints of the node's outputs (lfs, lgs: post-collision
// populations; lhn: the new history).  Out: adjoints of phi9, f and g (the
// collision paths only: phi's own dependence on f is added by the stream
// pass), h, and the node's dJ/dG.  With lfs = lgs = 0 it is also the adjoint
// of the history set-up at t = 0 (only the history outputs then matter).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void node_adjoint(const Phys<T>& P, const T phi9[9], const T f[9], const T g[9], const T h[5],
                             const T lfs[9], const T lgs[9], const T lhn[5], T lphi9[9], T lf[9], T lg[9],
                             T lh[5], T& lGx, T& lGy) {
  // ---------------- forward recomputation
  const T phi = phi9[0];
  const T gx = (phi9[1] - phi9[3]) * T(1.0 / 3.0) + ((phi9[5] - phi9[7]) + (phi9[8] - phi9[6])) * T(1.0 / 12.0);
  const T gy = (phi9[2] - phi9[4]) * T(1.0 / 3.0) + ((phi9[5] - phi9[7]) + (phi9[6] - phi9[8])) * T(1.0 / 12.0);
  const T lap = (((phi9[1] - phi) + (phi9[3] - phi)) + ((phi9[2] - phi) + (phi9[4] - phi))) * T(2.0 / 3.0) +
                (((phi9[5] - phi) + (phi9[7] - phi)) + ((phi9[6] - phi) + (phi9[8] - phi))) * T(1.0 / 6.0);
  const T pa = phi - P.phiA, pb = phi - P.phiB, pc = phi - P.phibar;
  const T mu = P.beta4 * pa * pb * pc - P.kappa * lap;
  const T lam = P.lam_coef * (P.phiA - phi) * pb;
  const T g2 = gx * gx + gy * gy;
  const T inv = inv_soft_norm(g2, P.n_delta);  // r = (g2^2 + delta^4)^(-1/4)
  const T nx_ = gx * inv, ny_ = gy * inv;
  const T Dx = gx - lam * nx_, Dy = gy - lam * ny_;
  const T rho = P.drho * pb + P.rhoB;
  const T rx = P.drho * gx, ry = P.drho * gy;
  const T mcx = -P.mob_drho * Dx, mcy = -P.mob_drho * Dy;
  const T Gs = P.gravity_mode == 0 ? T(1) : (P.gravity_mode == 1 ? rho : rho - P.rho_mean);
  const T Fx = mu * gx + Gs * P.gx, Fy = mu * gy + Gs * P.gy;
  const T ga = (g[1] + g[3]) + (g[2] + g[4]);
  const T gb = (g[5] + g[7]) + (g[6] + g[8]);
  const T g13 = g[1] - g[3], g24 = g[2] - g[4];
  const T gdx = (g[5] - g[7]) + (g[8] - g[6]);
  const T gdy = (g[5] - g[7]) + (g[6] - g[8]);
  const T irho = fdiv(T(1), rho);
  const T nxu = (g13 + gdx) + T(0.5) * Fx, nyu = (g24 + gdy) + T(0.5) * Fy;
  const T u = nxu * irho, v = nyu * irho;
  const T um = u * mcx + v * mcy, cA = u * mcx - v * mcy, cB = u * mcy + v * mcx;
  const T phu = phi * u, phv = phi * v;
  const T d_um = um - h[2], d_A = cA - h[3], d_B = cB - h[4];
  const T uu = u * u + v * v, ugr = u * rx + v * ry, uF = u * Fx + v * Fy;
  const T Z = rho * uu + um;
  const T s0 = T(-2.0 / 3.0) * Z;
  const T p = T(0.6) * ((ga + gb) + (T(0.5) + P.H) * ugr + s0 + P.K * (T(2) * uF + d_um));
  // viscous rates of moments 7, 8
  T s7 = P.sg[7], s8 = P.sg[8], dsn_drho = T(0), dsn_dphi = T(0);
  if (P.sg7_node | P.sg8_node) {
    const T frac = pb * P.inv_dphi;
    T snode;
    if (!P.visc_inverse) {
      const T muv = frac * (P.muA - P.muB) + P.muB;
      const T den = T(3) * muv + T(0.5) * rho;
      snode = rho / den;
      dsn_drho = T(3) * muv / (den * den);
      dsn_dphi = -T(3) * rho / (den * den) * (P.muA - P.muB) * P.inv_dphi;
    } else {
      const T inu = frac * (P.inuA - P.inuB) + P.inuB;
      const T den = T(3) + T(0.5) * inu;
      snode = inu / den;
      dsn_dphi = T(3) / (den * den) * (P.inuA - P.inuB) * P.inv_dphi;
    }
    if (P.sg7_node) s7 = snode;
    if (P.sg8_node) s8 = snode;
  }
  T mg[9];
  mmul(g, mg);
  const T E7 = cA + rho * (u * u - v * v);
  const T E8 = T(0.5) * cB + rho * u * v;
  const T Q7 = T(2.0 / 3.0) * (u * rx - v * ry) + T(2) * (u * Fx - v * Fy) + d_A;
  const T Q8 = T(1.0 / 3.0) * (u * ry + v * rx) + (u * Fy + v * Fx) + T(0.5) * d_B;

  // ---------------- reverse sweep
  T lphi = T(0), lu = T(0), lv = T(0), lrho = T(0), lFx = T(0), lFy = T(0), lrx = T(0), lry = T(0);
  T lum = T(0), lcA = T(0), lcB = T(0), lphu = T(0), lphv = T(0), luu = T(0), lugr = T(0), luF = T(0);
  T ld_phu = T(0), ld_phv = T(0), ld_um = T(0), ld_A = T(0), ld_B = T(0);
  T llam = T(0), lnx = T(0), lny = T(0), lmu = T(0), lgx = T(0), lgy = T(0);

  // f collision: fs = M^{-1}[m + s (eq - m) + (1 - s/2) src]
  {
    T a[9];
    mmul(lfs, a);
    T lmf[9];
    T leq[9], lsrc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const T lm = a[k] * T(inv_row_norm2(k));
      lmf[k] = (T(1) - P.sf[k]) * lm;
      leq[k] = P.sf[k] * lm;
      lsrc[k] = P.hf[k] * lm;
    }
    mtmul(lmf, lf);
    // eq = (phi, (-4 + 2 eta) phi, (4 - 3 eta) phi, phu, -phu, phv, -phv, 0, 0)
    lphi += leq[0] + (T(-4) + T(2) * P.eta) * leq[1] + (T(4) - T(3) * P.eta) * leq[2];
    lphu += leq[3] - leq[4];
    lphv += leq[5] - leq[6];
    // src: X = d(phi u) + lambda n / 3
    const T lXx = lsrc[3] - lsrc[4], lXy = lsrc[5] - lsrc[6];
    ld_phu += lXx;
    ld_phv += lXy;
    llam += (lXx * nx_ + lXy * ny_) * T(1.0 / 3.0);
    lnx += lXx * lam * T(1.0 / 3.0);
    lny += lXy * lam * T(1.0 / 3.0);
  }
  // g collision
  {
    T a[9];
    mmul(lgs, a);
    T lm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) lm[k] = a[k] * T(inv_row_norm2(k));
    T s[9];
#pragma unroll
    for (int k = 0; k < 7; ++k) s[k] = P.sg[k];
    s[7] = s7;
    s[8] = s8;
    T lmg[9], leq[9], lsrc[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      lmg[k] = (T(1) - s[k]) * lm[k];
      leq[k] = s[k] * lm[k];
      lsrc[k] = (T(1) - T(0.5) * s[k]) * lm[k];
    }
    mtmul(lmg, lg);
    // node-dependent rates: d m'/ds = eq - m - src / 2
    T lsn = T(0);
    if (P.sg7_node) lsn += lm[7] * (E7 - mg[7] - T(0.5) * Q7);
    if (P.sg8_node) lsn += lm[8] * (E8 - mg[8] - T(0.5) * Q8);
    lrho += lsn * dsn_drho;
    lphi += lsn * dsn_dphi;
    // equilibrium moments (deviation form): (0, E1, E2, E3, -E3, E5, -E5, E7, E8)
    const T lE1 = leq[1], lE2 = leq[2], lE3 = leq[3] - leq[4], lE5 = leq[5] - leq[6];
    const T lE7 = leq[7], lE8 = leq[8];
    // forcing moments: (Q0, Q1, Q2, Fx, -Fx, Fy, -Fy, Q7, Q8), Q0 = ugr, Q2 = -ugr - Q1
    const T lQ2 = lsrc[2];
    const T lQ1 = lsrc[1] - lQ2;
    lugr += lsrc[0] - lQ2;
    lFx += lsrc[3] - lsrc[4];
    lFy += lsrc[5] - lsrc[6];
    ld_um += T(3) * lQ1;
    luF += T(6) * lQ1;
    const T lQ7 = lsrc[7], lQ8 = lsrc[8];
    lu += lQ7 * (T(2.0 / 3.0) * rx + T(2) * Fx) + lQ8 * (T(1.0 / 3.0) * ry + Fy);
    lv += lQ7 * (T(-2.0 / 3.0) * ry - T(2) * Fy) + lQ8 * (T(1.0 / 3.0) * rx + Fx);
    lrx += lQ7 * T(2.0 / 3.0) * u + lQ8 * T(1.0 / 3.0) * v;
    lry += -lQ7 * T(2.0 / 3.0) * v + lQ8 * T(1.0 / 3.0) * u;
    lFx += T(2) * u * lQ7 + v * lQ8;
    lFy += -T(2) * v * lQ7 + u * lQ8;
    ld_A += lQ7;
    ld_B += T(0.5) * lQ8;
    // E1 = 6p + 3Z, E2 = -9p - 3Z
    T lp = T(6) * lE1 - T(9) * lE2;
    T lZ = T(3) * (lE1 - lE2);
    lrho += lE3 * u + lE5 * v + lE7 * (u * u - v * v) + lE8 * u * v;
    lu += lE3 * rho + lE7 * T(2) * rho * u + lE8 * rho * v;
    lv += lE5 * rho - lE7 * T(2) * rho * v + lE8 * rho * u;
    lcA += lE7;
    lcB += T(0.5) * lE8;
    // p = 0.6 (ga + gb + (1/2 + H) ugr + s0 + K (2 uF + d_um))
    const T lga = T(0.6) * lp;
    lugr += T(0.6) * (T(0.5) + P.H) * lp;
    const T ls0 = T(0.6) * lp;
    luF += T(1.2) * P.K * lp;
    ld_um += T(0.6) * P.K * lp;
    lZ += T(-2.0 / 3.0) * ls0;
    // Z = rho uu + um
    lrho += lZ * uu;
    luu += lZ * rho;
    lum += lZ;
    // pulled g through ga + gb (p)
#pragma unroll
    for (int i = 1; i < 9; ++i) lg[i] += lga;
  }
  // history outputs and derivatives d = chi - h
  lphu += lhn[0] + ld_phu;
  lphv += lhn[1] + ld_phv;
  lum += lhn[2] + ld_um;
  lcA += lhn[3] + ld_A;
  lcB += lhn[4] + ld_B;
  lh[0] = -ld_phu;
  lh[1] = -ld_phv;
  lh[2] = -ld_um;
  lh[3] = -ld_A;
  lh[4] = -ld_B;
  // uu, ugr, uF
  lu += T(2) * u * luu + rx * lugr + Fx * luF;
  lv += T(2) * v * luu + ry * lugr + Fy * luF;
  lrx += u * lugr;
  lry += v * lugr;
  lFx += u * luF;
  lFy += v * luF;
  // phi u, phi v
  lphi += u * lphu + v * lphv;
  lu += phi * lphu;
  lv += phi * lphv;
  // u.m, u mx - v my, u my + v mx
  lu += mcx * (lum + lcA) + mcy * lcB;
  lv += mcy * (lum - lcA) + mcx * lcB;
  const T lmcx = u * (lum + lcA) + v * lcB;
  const T lmcy = v * (lum - lcA) + u * lcB;
  // u = (g13 + gdx + Fx/2) / rho
  const T lnxu = lu * irho, lnyu = lv * irho;
  lrho -= (lu * nxu + lv * nyu) * irho * irho;
  lFx += T(0.5) * lnxu;
  lFy += T(0.5) * lnyu;
  lg[1] += lnxu;
  lg[3] -= lnxu;
  lg[2] += lnyu;
  lg[4] -= lnyu;
  lg[5] += lnxu + lnyu;
  lg[7] -= lnxu + lnyu;
  lg[8] += lnxu - lnyu;
  lg[6] += -lnxu + lnyu;
  // F = mu grad phi + Gs G
  lmu += lFx * gx + lFy * gy;
  lgx += lFx * mu;
  lgy += lFy * mu;
  const T lGs = lFx * P.gx + lFy * P.gy;
  lGx += lFx * Gs;
  lGy += lFy * Gs;
  if (P.gravity_mode != 0) lrho += lGs;
  // m^{phi C} = -(d rho/d phi) M D, grad rho, rho
  const T lDx = -P.mob_drho * lmcx, lDy = -P.mob_drho * lmcy;
  lgx += P.drho * lrx;
  lgy += P.drho * lry;
  lphi += P.drho * lrho;
  // D = grad phi - lambda n
  lgx += lDx;
  lgy += lDy;
  llam -= lDx * nx_ + lDy * ny_;
  lnx -= lDx * lam;
  lny -= lDy * lam;
  // n = grad phi r, r = (|grad phi|^4 + delta^4)^(-1/4), dr/dg = -|g|^2 g r^5:
  // dn/dg = r I - |g|^2 r^5 g g^T
  {
    const T r5 = inv * inv * inv * inv * inv;
    const T gl = (gx * lnx + gy * lny) * g2 * r5;
    lgx += inv * lnx - gx * gl;
    lgy += inv * lny - gy * gl;
  }
  // lambda, mu
  lphi += llam * P.lam_coef * ((P.phiA - phi) - pb);
  lphi += lmu * P.beta4 * (pb * pc + pa * pc + pa * pb);
  const T llap = -P.kappa * lmu;
  // stencils
  const T l4 = T(2.0 / 3.0) * llap, l8 = T(1.0 / 6.0) * llap;
  const T ax = lgx * T(1.0 / 3.0), ay = lgy * T(1.0 / 3.0);
  const T bx = lgx * T(1.0 / 12.0), by = lgy * T(1.0 / 12.0);
  lphi9[0] = lphi - T(4) * (l4 + l8);
  lphi9[1] = l4 + ax;
  lphi9[3] = l4 - ax;
  lphi9[2] = l4 + ay;
  lphi9[4] = l4 - ay;
  lphi9[5] = l8 + bx + by;
  lphi9[7] = l8 - bx - by;
  lphi9[8] = l8 + bx - by;
  lphi9[6] = l8 - bx + by;
}

// ---------------------------------------------------------------------------
// Kernels.  Adjoint planes use the population layout (row-interleaved, the
// handle's pitch); the extended phi adjoint is dense (nx + 2) x (ny + 2).
// ---------------------------------------------------------------------------
struct AdjBufs {
  void* lf;    // adjoint of f* (9 planes)
  void* lg;    // adjoint of g* (9 planes)
  void* lh;    // adjoint of the history (5 planes)
  void* lp9;   // per-node adjoint of the stencil phi values (9 planes)
  void* lfp;   // per-node adjoint of the pulled f through the collision (9 planes)
  void* lgp;   // per-node adjoint of the pulled g (9 planes)
  void* phi;   // forward phi(t) (1 plane)
  void* lext;  // adjoint of phi on the extended grid (dense)
  double* gpart;  // per-block dJ/dG partials (2 per block)
};

__host__ __device__ inline long long ext_index(int nx, int x, int y) {
  return (long long)(y + 1) * (nx + 2) + (x + 1);
}

template <typename T>
__global__ void k_adj_phi(const Phys<T> P, const T* __restrict__ fin, T* __restrict__ phi) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= P.nx) return;
  T v[9];
  pull9<PopPlain<T>>(fin, P, 0, x, y, v);
  phi[ix(P, 1, 0, x, y)] = sum9(v);
}

template <typename T>
__global__ void __launch_bounds__(ADJ_THREADS)
    k_adj_node(const Phys<T> P, const T* __restrict__ fin, const T* __restrict__ gin, const T* __restrict__ hist,
               const T* __restrict__ phi, const T* __restrict__ lf, const T* __restrict__ lg, T* __restrict__ lh,
               T* __restrict__ lp9, T* __restrict__ lfp, T* __restrict__ lgp, double* __restrict__ gpart,
               int hist_only) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  T gxs = T(0), gys = T(0);
  if (x < P.nx) {
    T phi9[9], f[9], g[9], h[5], lfs[9], lgs[9], lhn[5];
    const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
    for (int k = 0; k < 9; ++k) phi9[k] = phi_ext(P, phi, x + cx[k], y + cy[k]);
    pull9<PopPlain<T>>(fin, P, 0, x, y, f);
    pull9<PopPlain<T>>(gin, P, 1, x, y, g);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      h[k] = hist_only ? T(0) : hist[ix(P, 5, k, x, y)];
      lhn[k] = lh[ix(P, 5, k, x, y)];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      lfs[i] = hist_only ? T(0) : lf[ix(P, 9, i, x, y)];
      lgs[i] = hist_only ? T(0) : lg[ix(P, 9, i, x, y)];
    }
    T lphi9[9], lfo[9], lgo[9], lho[5], lGx = T(0), lGy = T(0);
    node_adjoint(P, phi9, f, g, h, lfs, lgs, lhn, lphi9, lfo, lgo, lho, lGx, lGy);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      lp9[ix(P, 9, k, x, y)] = lphi9[k];
      lfp[ix(P, 9, k, x, y)] = lfo[k];
      lgp[ix(P, 9, k, x, y)] = lgo[k];
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) lh[ix(P, 5, k, x, y)] = lho[k];
    gxs = lGx;
    gys = lGy;
  }
  // block sums of dJ/dG: within a warp in the arithmetic type, across warps
  // and blocks in double
  __shared__ double red[ADJ_THREADS / 32][2];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gxs += __shfl_down_sync(0xffffffffu, gxs, o);
    gys += __shfl_down_sync(0xffffffffu, gys, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[wid][0] = double(gxs);
    red[wid][1] = double(gys);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sx = 0.0, sy = 0.0;
    for (int w = 0; w < ADJ_THREADS / 32; ++w) {
      sx += red[w][0];
      sy += red[w][1];
    }
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
    gpart[2 * b] = sx;
    gpart[2 * b + 1] = sy;
  }
}

// Extended positions: x in [-wall_x, nx - 1 + wall_x], y likewise.
template <typename T>
__global__ void k_adj_gather(const Phys<T> P, const T* __restrict__ lp9, T* __restrict__ lext) {
  const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x) - P.wall_x;
  const int y = (int)blockIdx.y - P.wall_y;
  if (x >= P.nx + P.wall_x) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  T s = T(0);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    int sx = x - cx[k], sy = y - cy[k];  // the node whose stencil point k is (x, y)
    if (sx < 0 || sx >= P.nx) {
      if (P.wall_x) continue;
      sx = sx < 0 ? sx + P.nx : sx - P.nx;
    }
    if (sy < 0 || sy >= P.ny) {
      if (P.wall_y) continue;
      sy = sy < 0 ? sy + P.ny : sy - P.ny;
    }
    s += lp9[ix(P, 9, k, sx, sy)];
  }
  lext[ext_index(P.nx, x, y)] = s;
}

// Ghost rows beyond y walls, over the extended x range (one thread a column).
template <typename T>
__global__ void k_adj_fold_y(const Phys<T> P, const T* __restrict__ phi, T* __restrict__ lext) {
  const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x) - P.wall_x;
  if (x >= P.nx + P.wall_x || !P.wall_y) return;
  T d1, d2;
  const T lb = lext[ext_index(P.nx, x, -1)];
  wall_ghost_d(P, SIDE_BOTTOM, phi_xext(P, phi, x, 0), phi_xext(P, phi, x, 1), d1, d2);
  lext[ext_index(P.nx, x, 0)] += lb * d1;
  lext[ext_index(P.nx, x, 1)] += lb * d2;
  const T lt = lext[ext_index(P.nx, x, P.ny)];
  wall_ghost_d(P, SIDE_TOP, phi_xext(P, phi, x, P.ny - 1), phi_xext(P, phi, x, P.ny - 2), d1, d2);
  lext[ext_index(P.nx, x, P.ny - 1)] += lt * d1;
  lext[ext_index(P.nx, x, P.ny - 2)] += lt * d2;
}

// Ghost columns beyond x walls (one thread a row).
template <typename T>
__global__ void k_adj_fold_x(const Phys<T> P, const T* __restrict__ phi, T* __restrict__ lext) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  if (y >= P.ny || !P.wall_x) return;
  T d1, d2;
  const T ll = lext[ext_index(P.nx, -1, y)];
  wall_ghost_d(P, SIDE_LEFT, phi[ix(P, 1, 0, 0, y)], phi[ix(P, 1, 0, 1, y)], d1, d2);
  lext[ext_index(P.nx, 0, y)] += ll * d1;
  lext[ext_index(P.nx, 1, y)] += ll * d2;
  const T lr = lext[ext_index(P.nx, P.nx, y)];
  wall_ghost_d(P, SIDE_RIGHT, phi[ix(P, 1, 0, P.nx - 1, y)], phi[ix(P, 1, 0, P.nx - 2, y)], d1, d2);
  lext[ext_index(P.nx, P.nx - 1, y)] += lr * d1;
  lext[ext_index(P.nx, P.nx - 2, y)] += lr * d2;
}

// Reverse streaming into the adjoint of the previous post-collision state.
template <typename T>
__global__ void k_adj_stream(const Phys<T> P, const T* __restrict__ lfp, const T* __restrict__ lgp,
                             const T* __restrict__ lext, T* __restrict__ lf, T* __restrict__ lg) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= P.nx) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const int op[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int tx = x + cx[j], ty = y + cy[j];
    bool wall = false;
    if (tx < 0 || tx >= P.nx) { if (P.wall_x) wall = true; else tx = tx < 0 ? tx + P.nx : tx - P.nx; }
    if (ty < 0 || ty >= P.ny) { if (P.wall_y) wall = true; else ty = ty < 0 ? ty + P.ny : ty - P.ny; }
    const int rx = wall ? x : tx, ry = wall ? y : ty, k = wall ? op[j] : j;
    lf[ix(P, 9, j, x, y)] = lfp[ix(P, 9, k, rx, ry)] + lext[ext_index(P.nx, rx, ry)];
    lg[ix(P, 9, j, x, y)] = lgp[ix(P, 9, k, rx, ry)];
  }
}

// Seed: lambda of s_N for J = J(phi_N), phi_N = sum of the pulled f; dJ/dphi
// dense doubles [ny][nx].  g and history adjoints start at zero.
template <typename T>
__global__ void k_adj_seed(const Phys<T> P, const double* __restrict__ djdphi, T* __restrict__ lf,
                           T* __restrict__ lg, T* __restrict__ lh) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= P.nx) return;
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    int tx = x + cx[j], ty = y + cy[j];
    bool wall = false;
    if (tx < 0 || tx >= P.nx) { if (P.wall_x) wall = true; else tx = tx < 0 ? tx + P.nx : tx - P.nx; }
    if (ty < 0 || ty >= P.ny) { if (P.wall_y) wall = true; else ty = ty < 0 ? ty + P.ny : ty - P.ny; }
    const int rx = wall ? x : tx, ry = wall ? y : ty;
    lf[ix(P, 9, j, x, y)] = T(djdphi[(long long)ry * P.nx + rx]);
    lg[ix(P, 9, j, x, y)] = T(0);
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) lh[ix(P, 5, k, x, y)] = T(0);
}

// Adjoint of the initial state with respect to phi0: f*(s) holds the
// equilibria f^eq_i = c_i phi0 of the nodes it streams to, phi(0) = sum of
// the pulled f.  out (dense doubles) = sum_i c_i (pull of lambda_f + lext).
template <typename T>
__global__ void k_adj_init(const Phys<T> P, const T* __restrict__ lf, const T* __restrict__ lext,
                           double* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= P.nx) return;
  T v[9];
  pull9<PopPlain<T>>(lf, P, 0, x, y, v);
  const T e = P.eta;
  const T c0 = T(1) - T(5.0 / 9.0) * e, c1 = e * T(1.0 / 9.0), c2 = e * T(1.0 / 36.0);
  const T le = lext[ext_index(P.nx, x, y)];
  const T s = c0 * (v[0] + le) + c1 * ((v[1] + v[3]) + (v[2] + v[4]) + T(4) * le) +
              c2 * ((v[5] + v[7]) + (v[6] + v[8]) + T(4) * le);
  out[(long long)y * P.nx + x] = double(s);
}

// Sum of the per-block dJ/dG partials into acc[2].
template <typename T>
__global__ void k_adj_reduce(const double* __restrict__ part, long long nparts, double* __restrict__ acc) {
  __shared__ double red[256 / 32][2];
  double sx = 0.0, sy = 0.0;
  for (long long b = threadIdx.x; b < nparts; b += blockDim.x) {
    sx += part[2 * b];
    sy += part[2 * b + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_down_sync(0xffffffffu, sx, o);
    sy += __shfl_down_sync(0xffffffffu, sy, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[wid][0] = sx;
    red[wid][1] = sy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tx = 0.0, ty = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      tx += red[w][0];
      ty += red[w][1];
    }
    acc[0] += tx;
    acc[1] += ty;
  }
}

}  // namespace pflbm

