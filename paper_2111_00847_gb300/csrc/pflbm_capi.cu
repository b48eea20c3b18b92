// C-ABI of the GB300 phase-field lattice Boltzmann library (include/pflbm.h).
//
// Host side only: parameter validation, device memory (own cudaMalloc or a
// caller-supplied allocator), the per-run constants handed to the kernels,
// and the sequencing of launches on the handle's stream.  Every step of the
// method runs in the device kernels of pflbm_kernels.cuh.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pflbm.h"
#include "pflbm_launch.h"

using namespace pflbm;

struct lbm_handle {
  lbm_params prm;
  cudaStream_t stream = nullptr;
  lbm_allocator alloc{};
  bool have_alloc = false;
  int prec = LBM_FP64;
  int device = -1;       // the CUDA device current at lbm_create (all of the handle's memory is there)
  size_t esize = 8;      // bytes of the arithmetic type (history, macro planes)
  long long pop_bytes = 0;  // bytes of one population set (codec layout)
  int nx = 0, ny = 0, pitch = 0;
  long long plane = 0;
  void* pops[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [f|g][A|B]
  int cur = 0;
  void* hist = nullptr;
  void* phi_prev = nullptr;
  void* macro = nullptr;
  double* dstage = nullptr;
  int dstage_planes = 0;
  double* dpart = nullptr;
  double* ddiag = nullptr;
  int* derr = nullptr;  // device flag raised by a kernel whose bounded wait timed out
  bool use_tma = true;
  bool unit_rates = false;  // the rates the paper leaves at 1 are 1
  int nparts = 0;
  double diag[LBM_NDIAG] = {0};
  int64_t t = 0;
  int64_t bytes = 0;
  std::vector<std::pair<void*, size_t>> blocks;
  std::string err;
  // derived constants (double)
  double beta, kappa, lam_coef, drho, sf[9], sg[9], H;
  bool sg_node[9];
  double wa[4];
  double dv_r[2][2], dv_s[2], dv_c0;  // 16-bit deviation storage constants
  // discrete adjoint (created on first use)
  AdjBufs adj{};
  bool have_adj = false;
  double* gacc = nullptr;  // accumulated dJ/dG
  bool init_u_zero = true; // the last lbm_init_fields had u = 0
  // solid obstacles (lbm_set_solid): reflecting links per node and the phi /
  // mu_phi work planes of the obstacle passes
  uint16_t* dobs = nullptr;
  void* obs_planes = nullptr;
  int* dfill = nullptr;  // solid nodes next to fluid (dense indices)
  int nfill = 0;
  uint8_t* dnear = nullptr;  // per block of the TMA step's launch grid: reaches a solid node
  int near_box[4] = {0, 0, 0, 0};     // phi-plane region the passes fill for them (x_lo, x_hi, y_lo, y_hi)
  int near_box_mu[4] = {0, 0, 0, 0};  // the same for the mu_phi plane (Cahn-Hilliard)
  // y-slab of a larger grid (lbm_create_slab): rows [slab_y0, slab_y0 +
  // slab_own) of the global grid, held as local rows [ghost_lo, ghost_lo +
  // slab_own) between ghost rows that the halo exchange fills
  bool slab = false;
  int slab_y0 = 0, slab_own = 0, ghost_lo = 0, ghost_hi = 0;
};

static std::string g_create_error;

static int fail(lbm_handle* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_error = buf;
  return code;
}

#define CUDA_TRY(h, call)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail((h), e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s (%s)",    \
                  #call, cudaGetErrorString(e_), cudaGetErrorName(e_));                            \
  } while (0)

static void* dev_alloc(lbm_handle* h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  if (h->have_alloc) {
    p = h->alloc.alloc(bytes, (void*)h->stream, h->alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) {
    h->blocks.emplace_back(p, bytes);
    h->bytes += (int64_t)bytes;
  }
  return p;
}

static void dev_free(lbm_handle* h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->blocks.size(); ++i)
    if (h->blocks[i].first == p) {
      h->bytes -= (int64_t)h->blocks[i].second;
      h->blocks.erase(h->blocks.begin() + i);
      break;
    }
  if (h->have_alloc) h->alloc.free(p, (void*)h->stream, h->alloc.ctx);
  else cudaFree(p);
}

static double cos_deg(double th) { return th == 90.0 ? 0.0 : std::cos(th * 3.14159265358979323846 / 180.0); }

static int validate(const lbm_params* P) {
  if (!P) return fail(nullptr, LBM_EINVAL, "params is NULL");
  if (P->version != LBM_ABI_VERSION) return fail(nullptr, LBM_EINVAL, "params.version %d != %d", P->version, LBM_ABI_VERSION);
  if (P->nx < 3 || P->ny < 3) return fail(nullptr, LBM_EINVAL, "grid %d x %d: each side must be >= 3", P->nx, P->ny);
  const long long pitch = ((long long)P->nx + 2 * XPAD + 8 + 31) / 32 * 32;
  if (P->ny > 65535) return fail(nullptr, LBM_EINVAL, "ny = %d exceeds 65535", P->ny);
  if (pitch * P->ny >= (1LL << 31)) return fail(nullptr, LBM_EINVAL, "grid %d x %d too large (pitch*ny must be < 2^31)", P->nx, P->ny);
  if (P->precision != LBM_FP64 && P->precision != LBM_FP32 && P->precision != LBM_FP16_DEV &&
      P->precision != LBM_BF16_DEV)
    return fail(nullptr, LBM_EINVAL, "precision %d", P->precision);
  if (P->phase_model != LBM_AC && P->phase_model != LBM_CH) return fail(nullptr, LBM_EINVAL, "phase_model %d", P->phase_model);
  if (P->flux_model == LBM_CORRECTED) return fail(nullptr, LBM_EUNSUPPORTED, "flux_model CORRECTED is not built in this library");
  if (P->flux_model != LBM_PRESENT && P->flux_model != LBM_ORIGINAL) return fail(nullptr, LBM_EINVAL, "flux_model %d", P->flux_model);
  if (P->visc_law != LBM_LINEAR_MU && P->visc_law != LBM_INVERSE_NU) return fail(nullptr, LBM_EINVAL, "visc_law %d", P->visc_law);
  if (P->gravity_mode < 0 || P->gravity_mode > 2) return fail(nullptr, LBM_EINVAL, "gravity_mode %d", P->gravity_mode);
  if (P->bc[0] != P->bc[1] || P->bc[2] != P->bc[3]) return fail(nullptr, LBM_EINVAL, "opposite sides must share a boundary type");
  for (int s = 0; s < 4; ++s) {
    if (P->bc[s] != LBM_PERIODIC && P->bc[s] != LBM_WALL) return fail(nullptr, LBM_EINVAL, "bc[%d] = %d", s, P->bc[s]);
    if (!(P->theta_deg[s] >= 0.0 && P->theta_deg[s] <= 180.0)) return fail(nullptr, LBM_EINVAL, "theta_deg[%d] outside [0, 180]", s);
  }
  if (!(P->phiA > P->phiB)) return fail(nullptr, LBM_EINVAL, "phiA must exceed phiB");
  if (!(P->rhoA > 0 && P->rhoB > 0 && P->muA > 0 && P->muB > 0)) return fail(nullptr, LBM_EINVAL, "densities and viscosities must be positive");
  if (!(P->width > 0 && P->sigma >= 0 && P->mobility >= 0 && P->eta > 0)) return fail(nullptr, LBM_EINVAL, "width > 0, sigma >= 0, mobility >= 0, eta > 0 required");
  if (!(P->n_delta >= 0.0 && P->n_delta < 1.0)) return fail(nullptr, LBM_EINVAL, "n_delta must lie in [0, 1)");
  for (int k = 0; k < 9; ++k) {
    if (!std::isnan(P->s_f[k]) && !(P->s_f[k] > 0 && P->s_f[k] < 2)) return fail(nullptr, LBM_EINVAL, "s_f[%d] outside (0, 2)", k);
    if (!std::isnan(P->s_g[k]) && !(P->s_g[k] > 0 && P->s_g[k] < 2)) return fail(nullptr, LBM_EINVAL, "s_g[%d] outside (0, 2)", k);
  }
  const double amax = 4.0 / (P->width * (P->phiA - P->phiB));
  if (8.0 / 3.0 - amax * std::fabs(P->phiA + P->phiB) <= 0.0) return fail(nullptr, LBM_EINVAL, "interface width too small for the wetting root");
  if (P->precision == LBM_FP16_DEV) {
    // the FP16 deviation scale 2^(13 - ceil(log2 m)) and its inverse, which the
    // decode applies as an FP16 operand, must be powers of two FP16 holds
    // exactly: m = max(|phi_A|, |phi_B|) and m = max(rho_A, rho_B) in (2^-12, 2^28]
    const double pm = std::max(std::fabs(P->phiA), std::fabs(P->phiB)), rm = std::max(P->rhoA, P->rhoB);
    if (!(pm > 0x1p-12 && pm <= 0x1p28 && rm > 0x1p-12 && rm <= 0x1p28))
      return fail(nullptr, LBM_EINVAL, "FP16 deviation storage needs max |phi_A|, |phi_B| and max rho in (2^-12, 2^28]");
  }
  if (P->diag_every < 0) return fail(nullptr, LBM_EINVAL, "diag_every < 0");
  if (P->flags & ~LBM_FLAG_NO_TMA) return fail(nullptr, LBM_EINVAL, "unknown flags 0x%x", P->flags);
  return LBM_OK;
}

static void derive(lbm_handle* h) {
  const lbm_params& P = h->prm;
  const double dphi = P.phiA - P.phiB;
  // Eq. (3), Eq. (8), Eq. (10)
  h->beta = 12.0 * P.sigma / (P.width * dphi * dphi * dphi * dphi);
  h->kappa = 1.5 * P.sigma * P.width / (dphi * dphi);
  h->lam_coef = P.sigma > 0.0 ? std::sqrt(2.0 * h->beta / h->kappa) : 4.0 / (P.width * dphi);
  h->drho = (P.rhoA - P.rhoB) / dphi;
  // relaxation rates (Sec. 4): NaN -> default rule
  for (int k = 0; k < 9; ++k) {
    h->sf[k] = std::isnan(P.s_f[k]) ? ((k == 3 || k == 5) ? 1.0 / (3.0 * P.mobility / P.eta + 0.5) : 1.0) : P.s_f[k];
    h->sg_node[k] = std::isnan(P.s_g[k]) && (k == 7 || k == 8);
    h->sg[k] = std::isnan(P.s_g[k]) ? 1.0 : P.s_g[k];
  }
  h->unit_rates = true;
  for (int k = 0; k < 9; ++k) {
    if (k != 3 && k != 5 && h->sf[k] != 1.0) h->unit_rates = false;
    if ((k <= 3 || k == 5) && h->sg[k] != 1.0) h->unit_rates = false;
  }
  // App. C: H = (s_g^2 - s_g^0) / (9 s_g^0 s_g^2)
  h->H = (h->sg[2] - h->sg[0]) / (9.0 * h->sg[0] * h->sg[2]);
  for (int s = 0; s < 4; ++s) h->wa[s] = 4.0 * cos_deg(P.theta_deg[s]) / (P.width * dphi);
  // 16-bit deviation storage.  r: the ratios f_i / f_0 of a node at rest.
  // Allen-Cahn f^eq at u = 0 (Eq. (C.4)): f_0 = (1 - 5 eta / 9) phi, f_i =
  // w_i eta phi, so r_i = 9 w_i eta / (9 - 5 eta) (while f_0 keeps at least a
  // quarter of phi; else no reference).  Cahn-Hilliard f^eq at rest moves
  // only eta mu_phi (Eq. (C.3)), which vanishes in the bulk: r = 0.  g^eq at
  // rest (Eq. (C.2), g_0 stored minus rho0): g_0 = -(5/3) p, g_i = 3 w_i p,
  // so r_i = -9 w_i / 5.  Scales: 2^13 over the largest |phi| (rho) rounded
  // up to a power of two keeps FP16 deviations far below its 65504 limit
  // and above its subnormal range; BF16 has the FP32 exponent range.
  const bool ac_ref = P.phase_model == LBM_AC && 9.0 - 5.0 * P.eta >= 2.25;
  h->dv_r[0][0] = ac_ref ? P.eta / (9.0 - 5.0 * P.eta) : 0.0;
  h->dv_r[0][1] = ac_ref ? 0.25 * P.eta / (9.0 - 5.0 * P.eta) : 0.0;
  h->dv_c0 = 1.0 / (1.0 + 4.0 * h->dv_r[0][0] + 4.0 * h->dv_r[0][1]);
  h->dv_r[1][0] = -1.0 / 5.0;
  h->dv_r[1][1] = -1.0 / 20.0;
  const double phimax = std::max(std::fabs(P.phiA), std::fabs(P.phiB));
  const double rhomax = std::max(P.rhoA, P.rhoB);
  const bool half = P.precision == LBM_FP16_DEV;
  h->dv_s[0] = half ? std::ldexp(1.0, 13 - (int)std::ceil(std::log2(phimax))) : 1.0;
  h->dv_s[1] = half ? std::ldexp(1.0, 13 - (int)std::ceil(std::log2(rhomax))) : 1.0;
}

template <typename T>
static Phys<T> make_phys(const lbm_handle* h) {
  const lbm_params& Q = h->prm;
  Phys<T> P;
  std::memset(&P, 0, sizeof(P));
  P.nx = h->nx;
  P.ny = h->ny;
  P.pitch = h->pitch;
  P.plane = h->plane;
  P.wall_x = Q.bc[LBM_LEFT] == LBM_WALL;
  P.wall_y = Q.bc[LBM_BOTTOM] == LBM_WALL;
  P.gravity_mode = Q.gravity_mode;
  P.visc_inverse = Q.visc_law == LBM_INVERSE_NU;
  P.sg7_node = h->sg_node[7];
  P.sg8_node = h->sg_node[8];
  P.phiA = T(Q.phiA);
  P.phiB = T(Q.phiB);
  P.phibar = T(0.5 * (Q.phiA + Q.phiB));
  P.inv_dphi = T(1.0 / (Q.phiA - Q.phiB));
  P.beta4 = T(4.0 * h->beta);
  P.kappa = T(h->kappa);
  P.lam_coef = T(h->lam_coef);
  P.n_delta = T((Q.n_delta > 0.0 ? Q.n_delta : 5e-3) * (Q.phiA - Q.phiB) / Q.width);
  P.drho = T(h->drho);
  P.rhoB = T(Q.rhoB);
  P.rho_mean = T(0.5 * (Q.rhoA + Q.rhoB));
  P.mob_drho = Q.flux_model == LBM_PRESENT ? T(h->drho * Q.mobility) : T(0);
  P.muA = T(Q.muA);
  P.muB = T(Q.muB);
  P.inuA = T(Q.rhoA / Q.muA);
  P.inuB = T(Q.rhoB / Q.muB);
  P.gx = T(Q.gx);
  P.gy = T(Q.gy);
  P.eta = T(Q.eta);
  P.H = T(h->H);
  P.K = T(1.0 / 3.0);
  for (int k = 0; k < 9; ++k) {
    P.sf[k] = T(h->sf[k]);
    P.hf[k] = T(1.0 - 0.5 * h->sf[k]);
    P.sg[k] = T(h->sg[k]);
    P.hg[k] = T(1.0 - 0.5 * h->sg[k]);
  }
  for (int s = 0; s < 4; ++s) P.wa[s] = T(h->wa[s]);
  for (int set = 0; set < 2; ++set) {
    P.dv_r[set][0] = T(h->dv_r[set][0]);
    P.dv_r[set][1] = T(h->dv_r[set][1]);
    P.dv_s[set] = T(h->dv_s[set]);
    P.dv_is[set] = T(1.0 / h->dv_s[set]);
  }
  P.dv_c0 = T(h->dv_c0);
  P.obs = h->dobs;
  P.obs_fill = h->dfill;
  P.obs_nfill = h->nfill;
  P.obs_near = h->dnear;
  for (int k = 0; k < 4; ++k) P.obs_box[k] = h->near_box[k], P.obs_box_mu[k] = h->near_box_mu[k];
  P.diag_y0 = h->slab ? h->ghost_lo : 0;
  P.diag_y1 = h->slab ? h->ghost_lo + h->slab_own : h->ny;
  return P;
}

// ---------------------------------------------------------------------------
// Typed operations (T = float or double)
// ---------------------------------------------------------------------------
template <typename T>
static Bufs<T> bufs_now(lbm_handle* h) {
  Bufs<T> B;
  std::memset(&B, 0, sizeof(B));
  B.fin = h->pops[0][h->cur];
  B.gin = h->pops[1][h->cur];
  B.fout = h->pops[0][1 - h->cur];
  B.gout = h->pops[1][1 - h->cur];
  B.hist = (T*)h->hist;
  B.macro = (T*)h->macro;
  return B;
}

static int ensure_stage(lbm_handle* h, int planes) {
  if (h->dstage_planes >= planes) return LBM_OK;
  if (h->dstage) dev_free(h, h->dstage);
  h->dstage = (double*)dev_alloc(h, (size_t)planes * h->nx * h->ny * sizeof(double));
  h->dstage_planes = h->dstage ? planes : 0;
  if (!h->dstage) return fail(h, LBM_ENOMEM, "staging buffer of %d planes", planes);
  return LBM_OK;
}

static int ensure_macro(lbm_handle* h) {
  if (h->macro) return LBM_OK;
  h->macro = dev_alloc(h, (size_t)NMACRO * h->plane * h->esize);
  if (!h->macro) return fail(h, LBM_ENOMEM, "macro planes");
  return LBM_OK;
}

// A kernel whose bounded wait timed out raised *derr; report it once the
// stream has been synchronised.
static int check_device_flag(lbm_handle* h) {
  int flag = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&flag, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (flag) {
    cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    return fail(h, LBM_ECUDA, "a step kernel gave up waiting for its staged rows (results since the last check are invalid)");
  }
  return LBM_OK;
}

// One pass of the fused kernel in a mode, or, with solid obstacles, the
// obstacle passes (pflbm_obstacle.cuh).
template <class C>
static cudaError_t launch_mode(lbm_handle* h, int mode, const Phys<typename C::value_t>& P,
                               const Bufs<typename C::value_t>& B) {
  using T = typename C::value_t;
  if (!h->dobs) return launch_march<C>(h->prm.phase_model, mode, P, B, h->stream);
  T* phis = (T*)h->obs_planes;
  return launch_obs<C>(h->prm.phase_model, mode, P, B, phis, phis + h->plane, h->unit_rates, h->derr, h->use_tma,
                       h->stream);
}

template <class C>
static int run_macro(lbm_handle* h) {
  using T = typename C::value_t;
  int rc = ensure_macro(h);
  if (rc) return rc;
  const Phys<T> P = make_phys<T>(h);
  Bufs<T> B = bufs_now<T>(h);
  B.macro = (T*)h->macro;
  CUDA_TRY(h, launch_mode<C>(h, MODE_MACRO, P, B));
  return LBM_OK;
}

template <class C>
static int run_diag(lbm_handle* h) {
  using T = typename C::value_t;
  int rc = run_macro<C>(h);
  if (rc) return rc;
  const Phys<T> P = make_phys<T>(h);
  CUDA_TRY(h, launch_diag<T>(P, (const T*)h->macro, (const T*)h->phi_prev, h->dpart, h->nparts, h->ddiag, h->stream));
  double r[DIAG_FIELDS];
  CUDA_TRY(h, cudaMemcpyAsync(r, h->ddiag, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  int rc2 = check_device_flag(h);
  if (rc2) return rc2;
  const double n = r[5];
  h->diag[0] = (double)h->t;
  h->diag[1] = r[0];
  h->diag[2] = n > 0 ? std::sqrt(r[1] / n) : 0.0;
  h->diag[3] = n > 0 ? std::sqrt(r[2] / n) : 0.0;
  h->diag[4] = r[3];
  h->diag[5] = r[4];
  h->diag[6] = n;
  h->diag[7] = 0.0;
  return LBM_OK;
}

template <class C>
static int do_step(lbm_handle* h, int64_t n) {
  using T = typename C::value_t;
  const Phys<T> P = make_phys<T>(h);
  const int de = h->prm.diag_every;
  for (int64_t s = 0; s < n; ++s) {
    // a slab's ghost rows are stale until the next halo exchange, so its
    // diagnostics are taken on request (lbm_fields LBM_DIAG) after it; the
    // step still records phi(t-1) for their S_m
    const bool record = de > 0 && ((h->t + 1) % de == 0);
    const bool due = record && !h->slab;
    Bufs<T> B = bufs_now<T>(h);
    B.phi_prev = record ? (T*)h->phi_prev : nullptr;
    cudaError_t e = cudaErrorNotSupported;
    if (h->dobs)
      e = launch_mode<C>(h, MODE_STEP, P, B);
    else if (h->use_tma && h->prm.phase_model == LBM_AC)
      e = launch_step_tma<C>(P, B, h->derr, h->unit_rates, h->stream);
    else if (h->use_tma && h->prm.phase_model == LBM_CH)
      e = launch_step_tma_ch<C>(P, B, h->derr, h->unit_rates, h->stream);
    if (e == cudaErrorNotSupported) e = launch_march<C>(h->prm.phase_model, MODE_STEP, P, B, h->stream);
    CUDA_TRY(h, e);
    h->cur ^= 1;
    h->t += 1;
    if (due) {
      int rc = run_diag<C>(h);
      if (rc) return rc;
      if (h->diag[5] > 0 || !(h->diag[4] <= 0.4))
        return fail(h, LBM_EUNSTABLE, "unstable at t=%lld: %g non-finite nodes, max|u| = %g",
                    (long long)h->t, h->diag[5], h->diag[4]);
    }
  }
  CUDA_TRY(h, cudaGetLastError());
  return LBM_OK;
}

// Plain arithmetic-type scratch of nine planes (deviation storage: the
// pulled-layout equilibria and imported populations before encoding).
// Allocated per use and released by the caller, so that a run with 16-bit
// storage keeps its smaller footprint between such calls.
template <typename T>
static T* alloc_plain_pops(lbm_handle* h, int sets) {
  return (T*)dev_alloc(h, (size_t)sets * 9 * h->plane * sizeof(T));
}

template <class C>
static int do_init(lbm_handle* h, const double* phi, const double* ux, const double* uy, const double* p) {
  using T = typename C::value_t;
  const long long N = (long long)h->nx * h->ny;
  const int planes = 1 + (ux ? 1 : 0) + (uy ? 1 : 0) + (p ? 1 : 0);
  int rc = ensure_stage(h, planes);
  if (rc) return rc;
  const Phys<T> P = make_phys<T>(h);
  Bufs<T> B = bufs_now<T>(h);
  double* d = h->dstage;
  CUDA_TRY(h, cudaMemcpyAsync(d, phi, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  B.iphi = d;
  d += N;
  if (ux) { CUDA_TRY(h, cudaMemcpyAsync(d, ux, N * sizeof(double), cudaMemcpyHostToDevice, h->stream)); B.iux = d; d += N; }
  if (uy) { CUDA_TRY(h, cudaMemcpyAsync(d, uy, N * sizeof(double), cudaMemcpyHostToDevice, h->stream)); B.iuy = d; d += N; }
  if (p) { CUDA_TRY(h, cudaMemcpyAsync(d, p, N * sizeof(double), cudaMemcpyHostToDevice, h->stream)); B.ip = d; d += N; }
  if constexpr (!C::dev) {
    // equilibria per node into the spare buffers, then scatter to the pull layout
    CUDA_TRY(h, launch_mode<C>(h, MODE_INIT, P, B));
    CUDA_TRY(h, launch_unstream<T>(P, (const T*)h->pops[0][1 - h->cur], (T*)h->pops[0][h->cur], h->stream));
    CUDA_TRY(h, launch_unstream<T>(P, (const T*)h->pops[1][1 - h->cur], (T*)h->pops[1][h->cur], h->stream));
  } else {
    // equilibria per node into plain scratch, then encode node by node
    T* scratch = alloc_plain_pops<T>(h, 2);
    if (!scratch) return fail(h, LBM_ENOMEM, "scratch for the initial populations");
    T* gs = scratch + 9 * h->plane;
    B.fout = scratch;
    B.gout = gs;
    cudaError_t e = launch_mode<C>(h, MODE_INIT, P, B);
    if (e == cudaSuccess) e = launch_restream<C>(P, scratch, h->pops[0][h->cur], 0, h->stream);
    if (e == cudaSuccess) e = launch_restream<C>(P, gs, h->pops[1][h->cur], 1, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, scratch);
    CUDA_TRY(h, e);
  }
  // history := chi(0), and phi(t-1) := phi(0)
  Bufs<T> Bh = bufs_now<T>(h);
  Bh.phi_prev = (T*)h->phi_prev;
  CUDA_TRY(h, launch_mode<C>(h, MODE_HIST, P, Bh));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->t = 0;
  std::memset(h->diag, 0, sizeof(h->diag));
  return LBM_OK;
}

struct Region {
  int x0, y0, w, h;
};

// planes [k0, k0 + planes) of a set of NP interleaved planes -> host doubles
template <typename T>
static int export_planes(lbm_handle* h, const T* src, int NP, int k0, int planes, double add0, double* out,
                         Region r) {
  int rc = ensure_stage(h, 1);
  if (rc) return rc;
  const Phys<T> P = make_phys<T>(h);
  const long long N = (long long)r.w * r.h;
  for (int k = 0; k < planes; ++k) {
    CUDA_TRY(h, launch_export<T>(P, src, NP, k0 + k, h->dstage, k == 0 ? add0 : 0.0, r.x0, r.y0, r.w, r.h,
                                 h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(out + k * N, h->dstage, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

// host doubles -> all NP planes of an interleaved set (plane 0 minus sub0)
template <typename T>
static int import_planes(lbm_handle* h, const double* in, int NP, double sub0, T* dst) {
  int rc = ensure_stage(h, 1);
  if (rc) return rc;
  const Phys<T> P = make_phys<T>(h);
  const long long N = (long long)h->nx * h->ny;
  for (int k = 0; k < NP; ++k) {
    CUDA_TRY(h, cudaMemcpyAsync(h->dstage, in + k * N, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, launch_import<T>(P, h->dstage, dst, NP, k, k == 0 ? sub0 : 0.0, h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

// deviation storage: pulled populations of a region, decoded, -> host
template <class C>
static int export_pulled(lbm_handle* h, int set, double* out, Region r, double* stage) {
  using T = typename C::value_t;
  const Phys<T> P = make_phys<T>(h);
  const long long N = (long long)r.w * r.h;
  for (int k = 0; k < 9; ++k) {
    CUDA_TRY(h, launch_pull_export<C>(P, h->pops[set][h->cur], set, k, stage,
                                      (k == 0 && set == 1) ? h->prm.rho0 : 0.0, r.x0, r.y0, r.w, r.h,
                                      h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(out + k * N, stage, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

template <class C>
static int do_fields(lbm_handle* h, int which, double* out, Region reg) {
  using T = typename C::value_t;
  const Phys<T> P = make_phys<T>(h);
  switch (which) {
    case LBM_F_POP:
    case LBM_G_POP: {
      const int s = which == LBM_F_POP ? 0 : 1;
      if constexpr (C::dev) {
        int rc = ensure_stage(h, 1);
        if (rc) return rc;
        return export_pulled<C>(h, s, out, reg, h->dstage);
      }
      T* scratch = (T*)h->pops[s][1 - h->cur];
      CUDA_TRY(h, launch_pull<T>(P, (const T*)h->pops[s][h->cur], scratch, h->stream));
      return export_planes<T>(h, scratch, 9, 0, 9, s == 1 ? h->prm.rho0 : 0.0, out, reg);
    }
    case LBM_HIST:
      return export_planes<T>(h, (const T*)h->hist, 5, 0, 5, 0.0, out, reg);
    case LBM_DIAG: {
      int rc = run_diag<C>(h);
      if (rc) return rc;
      std::memcpy(out, h->diag, sizeof(h->diag));
      return LBM_OK;
    }
    default:
      break;
  }
  int plane;
  switch (which) {
    case LBM_PHI: plane = MAC_PHI; break;
    case LBM_UX: plane = MAC_UX; break;
    case LBM_UY: plane = MAC_UY; break;
    case LBM_P: plane = MAC_P; break;
    case LBM_RHO: plane = MAC_RHO; break;
    case LBM_MU: plane = MAC_MU; break;
    case LBM_MCX: plane = MAC_MCX; break;
    case LBM_MCY: plane = MAC_MCY; break;
    default: return fail(h, LBM_EINVAL, "unknown field selector %d", which);
  }
  int rc = run_macro<C>(h);
  if (rc) return rc;
  return export_planes<T>(h, (const T*)h->macro, NMACRO, plane, 1, 0.0, out, reg);
}

template <class C>
static int do_set_fields(lbm_handle* h, int which, const double* in) {
  using T = typename C::value_t;
  const Phys<T> P = make_phys<T>(h);
  switch (which) {
    case LBM_F_POP:
    case LBM_G_POP: {
      const int s = which == LBM_F_POP ? 0 : 1;
      if constexpr (C::dev) {
        T* scratch = alloc_plain_pops<T>(h, 1);
        if (!scratch) return fail(h, LBM_ENOMEM, "scratch for the imported populations");
        int rc = import_planes<T>(h, in, 9, s == 1 ? h->prm.rho0 : 0.0, scratch);
        cudaError_t e = cudaSuccess;
        if (!rc) e = launch_restream<C>(P, scratch, h->pops[s][h->cur], s, h->stream);
        if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        dev_free(h, scratch);
        if (rc) return rc;
        CUDA_TRY(h, e);
        return LBM_OK;
      }
      T* scratch = (T*)h->pops[s][1 - h->cur];
      int rc = import_planes<T>(h, in, 9, s == 1 ? h->prm.rho0 : 0.0, scratch);
      if (rc) return rc;
      CUDA_TRY(h, launch_unstream<T>(P, scratch, (T*)h->pops[s][h->cur], h->stream));
      CUDA_TRY(h, cudaStreamSynchronize(h->stream));
      return LBM_OK;
    }
    case LBM_HIST:
      return import_planes<T>(h, in, 5, 0.0, (T*)h->hist);
    default:
      return fail(h, LBM_EINVAL, "field %d cannot be set", which);
  }
}

// Run the codec-templated operation that matches the handle's storage.
#define PFLBM_DISPATCH(h, fn, ...)                                         \
  switch ((h)->prec) {                                                     \
    case LBM_FP64: return fn<PopPlain<double>>(__VA_ARGS__);               \
    case LBM_FP32: return fn<PopPlain<float>>(__VA_ARGS__);                \
    case LBM_FP16_DEV: return fn<PopDev<__half>>(__VA_ARGS__);             \
    default: return fn<PopDev<__nv_bfloat16>>(__VA_ARGS__);                \
  }

// Solid obstacles on the TMA steps: which blocks of the step's launch grid
// reach a solid node (within 3 nodes of their rows and columns: the pulls
// and the phi ring, whose nodes pull from one node further, reach 3), and
// the regions of the planes the per-step passes fill for those blocks.  The
// Allen-Cahn blocks read phi up to 1 node beyond their rows and columns and
// the phi pass forms its fill itself, so phi covers them widened by 2.  The
// Cahn-Hilliard blocks read phi up to 2 nodes beyond and mu_phi up to 1;
// the mu_phi fill reads mu_phi one node further and mu_phi reads phi one node
// further, so mu_phi covers them widened by 2 and phi widened by 3.  Blocks
// away from obstacles run the plain step's path.  Periodic sides wrap; a
// region that wraps takes the whole extent of its direction.
template <class C>
static int build_near_map(lbm_handle* h, const uint8_t* solid, bool ch) {
  int tbx = 0, seg = 0;
  if (ch) tma_ch_step_grid<C>(h->nx, h->ny, &tbx, &seg);
  else tma_step_grid<C>(h->nx, h->ny, &tbx, &seg);
  const int nx = h->nx, ny = h->ny;
  const bool px = h->prm.bc[LBM_LEFT] == LBM_PERIODIC, py = h->prm.bc[LBM_BOTTOM] == LBM_PERIODIC;
  const int gx = (nx + tbx - 1) / tbx, gy = (ny + seg - 1) / seg;
  std::vector<uint8_t> nearv((size_t)gx * gy, 0);
  // a block is near when a solid node lies in its rows and columns widened by
  // 3; mark, for every solid node, the blocks whose widened range holds it:
  // the blocks of the columns (rows) c - 3 .. c + 3, clamped at walls and
  // wrapped at periodic sides (a ragged last strip or a short segment can
  // sit wholly inside that range, so every position is looked at)
  auto blocks_of = [](int c, int n, int width, bool periodic, int out[7]) {
    int k = 0;
    for (int d = -3; d <= 3; ++d) {
      int cc = c + d;
      if (cc < 0 || cc >= n) cc = periodic ? ((cc % n) + n) % n : std::min(std::max(cc, 0), n - 1);
      const int b = cc / width;
      bool seen = false;
      for (int i = 0; i < k; ++i) seen = seen || out[i] == b;
      if (!seen) out[k++] = b;
    }
    return k;
  };
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (!solid[(size_t)y * nx + x]) continue;
      int bxs[7], bys[7];
      const int kx = blocks_of(x, nx, tbx, px, bxs), ky = blocks_of(y, ny, seg, py, bys);
      for (int j = 0; j < ky; ++j)
        for (int i = 0; i < kx; ++i) nearv[(size_t)bys[j] * gx + bxs[i]] = 1;
    }
  // the union of the near blocks' regions widened by `wd`
  auto box_of = [&](int wd, int box[4]) {
    int bx0 = nx, bx1 = 0, by0 = ny, by1 = 0;
    bool xwrap = false, ywrap = false;
    for (int by = 0; by < gy; ++by)
      for (int bx = 0; bx < gx; ++bx) {
        if (!nearv[(size_t)by * gx + bx]) continue;
        const int x0 = bx * tbx, x1 = std::min(x0 + tbx, nx), y0 = by * seg, y1 = std::min(y0 + seg, ny);
        xwrap = xwrap || (px && (x0 - wd < 0 || x1 + wd > nx));
        ywrap = ywrap || (py && (y0 - wd < 0 || y1 + wd > ny));
        bx0 = std::min(bx0, std::max(x0 - wd, 0)), bx1 = std::max(bx1, std::min(x1 + wd, nx));
        by0 = std::min(by0, std::max(y0 - wd, 0)), by1 = std::max(by1, std::min(y1 + wd, ny));
      }
    box[0] = xwrap ? 0 : bx0;
    box[1] = xwrap ? nx : bx1;
    box[2] = ywrap ? 0 : by0;
    box[3] = ywrap ? ny : by1;
  };
  box_of(ch ? 3 : 2, h->near_box);
  box_of(2, h->near_box_mu);
  h->dnear = (uint8_t*)dev_alloc(h, nearv.size());
  if (!h->dnear) return fail(h, LBM_ENOMEM, "obstacle block map");
  CUDA_TRY(h, cudaMemcpyAsync(h->dnear, nearv.data(), nearv.size(), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));  // nearv is released on return
  return LBM_OK;
}

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
extern "C" {

static int create_impl(const lbm_params* params, void* stream, const lbm_allocator* alloc, lbm_handle** out);

int lbm_create(const lbm_params* params, void* stream, const lbm_allocator* alloc, lbm_handle** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(params);
  if (rc) return rc;
  return create_impl(params, stream, alloc, out);
}

}  // extern "C"

static int create_impl(const lbm_params* params, void* stream, const lbm_allocator* alloc, lbm_handle** out) {
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(nullptr, LBM_EINVAL, "allocator needs alloc and free");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(nullptr, LBM_ECUDA, "no CUDA device available");
  }
  lbm_handle* h = new (std::nothrow) lbm_handle();
  if (!h) return fail(nullptr, LBM_ENOMEM, "host allocation");
  h->prm = *params;
  h->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(nullptr, LBM_ECUDA, "cannot query the current CUDA device");
  }
  if (alloc) {
    h->alloc = *alloc;
    h->have_alloc = true;
  }
  h->prec = params->precision;
  h->use_tma = (params->flags & LBM_FLAG_NO_TMA) == 0;
  const bool dev16 = h->prec == LBM_FP16_DEV || h->prec == LBM_BF16_DEV;
  h->esize = h->prec == LBM_FP64 ? 8 : 4;
  h->nx = params->nx;
  h->ny = params->ny;
  // rows carry XPAD pad elements per side; the pitch leaves room for a
  // 16-byte rounded bulk copy of the last strip's segment (up to 7 more
  // elements for 2-byte planes, 3 for 4-byte ones)
  h->pitch = (h->nx + 2 * XPAD + (dev16 ? 8 : 4) + 31) / 32 * 32;
  h->plane = (long long)h->pitch * h->ny;
  derive(h);
  const size_t pl = (size_t)h->plane * h->esize;
  h->pop_bytes = (dev16 ? pop_row_bytes<PopDev<__half>>(h->pitch) : 9LL * h->pitch * (long long)h->esize) * h->ny;
  bool ok = true;
  for (int s = 0; s < 2; ++s)
    for (int b = 0; b < 2; ++b) ok = ok && (h->pops[s][b] = dev_alloc(h, (size_t)h->pop_bytes));
  ok = ok && (h->hist = dev_alloc(h, 5 * pl));
  ok = ok && (h->phi_prev = dev_alloc(h, pl));
  const long long N = (long long)h->nx * h->ny;
  h->nparts = (int)std::min<long long>((N + DIAG_THREADS - 1) / DIAG_THREADS, 152 * 8);
  ok = ok && (h->dpart = (double*)dev_alloc(h, (size_t)h->nparts * DIAG_FIELDS * sizeof(double)));
  ok = ok && (h->ddiag = (double*)dev_alloc(h, DIAG_FIELDS * sizeof(double)));
  ok = ok && (h->derr = (int*)dev_alloc(h, sizeof(int)));
  if (!ok) {
    std::string msg = "device allocation of " + std::to_string(h->bytes) + " bytes failed";
    lbm_destroy(h);
    return fail(nullptr, LBM_ENOMEM, "%s", msg.c_str());
  }
  // zero the state so that a step before lbm_init_fields is well defined
  for (auto& b : h->blocks) cudaMemsetAsync(b.first, 0, b.second, h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    lbm_destroy(h);
    return fail(nullptr, LBM_ECUDA, "initial memset: %s", cudaGetErrorString(e));
  }
  *out = h;
  return LBM_OK;
}

extern "C" {

int lbm_init_fields(lbm_handle* h, const double* phi, const double* ux, const double* uy, const double* p) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!phi) return fail(h, LBM_EINVAL, "phi is NULL");
  h->init_u_zero = !ux && !uy;
  PFLBM_DISPATCH(h, do_init, h, phi, ux, uy, p);
}

int lbm_step(lbm_handle* h, int64_t nsteps) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (nsteps < 0) return fail(h, LBM_EINVAL, "nsteps < 0");
  if (h->slab && nsteps > 1)
    return fail(h, LBM_EINVAL, "a y-slab advances one step per call: exchange its halos between steps");
  PFLBM_DISPATCH(h, do_step, h, nsteps);
}

int lbm_fields_region(lbm_handle* h, int32_t which, int32_t x0, int32_t y0, int32_t w, int32_t hgt,
                      double* out) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  if (x0 < 0 || y0 < 0 || w < 1 || hgt < 1 || (long long)x0 + w > h->nx || (long long)y0 + hgt > h->ny)
    return fail(h, LBM_EINVAL, "region [%d,%d)x[%d,%d) outside the %d x %d grid", x0, x0 + w, y0, y0 + hgt,
                h->nx, h->ny);
  const Region r{x0, y0, w, hgt};
  PFLBM_DISPATCH(h, do_fields, h, which, out, r);
}

int lbm_fields(lbm_handle* h, int32_t which, double* out) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  return lbm_fields_region(h, which, 0, 0, h->nx, h->ny, out);
}

int lbm_set_fields(lbm_handle* h, int32_t which, const double* in) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!in) return fail(h, LBM_EINVAL, "in is NULL");
  PFLBM_DISPATCH(h, do_set_fields, h, which, in);
}

int lbm_set_solid(lbm_handle* h, const uint8_t* solid) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (h->slab) return fail(h, LBM_EUNSUPPORTED, "solid obstacles are not supported on a y-slab");
  long long nsolid = 0;
  const long long N = (long long)h->nx * h->ny;
  if (solid)
    for (long long n = 0; n < N; ++n) nsolid += solid[n] != 0;
  if (h->dobs) {  // drop the previous mask's buffers
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    dev_free(h, h->dobs);
    dev_free(h, h->obs_planes);
    dev_free(h, h->dfill);
    dev_free(h, h->dnear);
    h->dobs = nullptr;
    h->obs_planes = nullptr;
    h->dfill = nullptr;
    h->dnear = nullptr;
    h->nfill = 0;
  }
  if (nsolid == 0) return LBM_OK;  // no obstacles: the fused kernels
  // solid nodes with a fluid node among their 8 neighbours (periodic sides
  // wrap; nothing lies beyond a wall)
  std::vector<int> fill;
  {
    const int nx = h->nx, ny = h->ny;
    const bool wx = h->prm.bc[LBM_LEFT] == LBM_WALL, wy = h->prm.bc[LBM_BOTTOM] == LBM_WALL;
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        if (!solid[(long long)y * nx + x]) continue;
        bool near = false;
        for (int dy = -1; dy <= 1 && !near; ++dy)
          for (int dx = -1; dx <= 1 && !near; ++dx) {
            int xn = x + dx, yn = y + dy;
            if (xn < 0 || xn >= nx) { if (wx) continue; xn = (xn + nx) % nx; }
            if (yn < 0 || yn >= ny) { if (wy) continue; yn = (yn + ny) % ny; }
            near = !solid[(long long)yn * nx + xn];
          }
        if (near) fill.push_back(y * nx + x);
      }
  }
  h->dobs = (uint16_t*)dev_alloc(h, (size_t)N * sizeof(uint16_t));
  h->obs_planes = dev_alloc(h, 2 * (size_t)h->plane * h->esize);
  h->dfill = (int*)dev_alloc(h, std::max<size_t>(fill.size(), 1) * sizeof(int));
  if (!h->dobs || !h->obs_planes || !h->dfill) {
    dev_free(h, h->dobs);
    dev_free(h, h->obs_planes);
    dev_free(h, h->dfill);
    h->dobs = nullptr;
    h->obs_planes = nullptr;
    h->dfill = nullptr;
    return fail(h, LBM_ENOMEM, "obstacle planes");
  }
  h->nfill = (int)fill.size();
  CUDA_TRY(h, cudaMemsetAsync(h->obs_planes, 0, 2 * (size_t)h->plane * h->esize, h->stream));
  if (!fill.empty())
    CUDA_TRY(h, cudaMemcpyAsync(h->dfill, fill.data(), fill.size() * sizeof(int), cudaMemcpyHostToDevice,
                                h->stream));
  // the byte mask goes through the staging buffer (N bytes <= N doubles)
  int rc = ensure_stage(h, 1);
  if (rc) return rc;
  CUDA_TRY(h, cudaMemcpyAsync(h->dstage, solid, (size_t)N, cudaMemcpyHostToDevice, h->stream));
  if (h->prec == LBM_FP64) {
    const Phys<double> P = make_phys<double>(h);
    CUDA_TRY(h, launch_obs_links<double>(P, (const unsigned char*)h->dstage, h->dobs, h->stream));
  } else {
    const Phys<float> P = make_phys<float>(h);
    CUDA_TRY(h, launch_obs_links<float>(P, (const unsigned char*)h->dstage, h->dobs, h->stream));
  }
  if (h->use_tma && h->nx >= 4 * XPAD) {
    const bool ch = h->prm.phase_model == LBM_CH;
    switch (h->prec) {
      case LBM_FP64: rc = build_near_map<PopPlain<double>>(h, solid, ch); break;
      case LBM_FP32: rc = build_near_map<PopPlain<float>>(h, solid, ch); break;
      case LBM_FP16_DEV: rc = build_near_map<PopDev<__half>>(h, solid, ch); break;
      default: rc = build_near_map<PopDev<__nv_bfloat16>>(h, solid, ch); break;
    }
    if (rc) return rc;
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

}  // extern "C"

// One thread waits, with the step kernels' bounded wait, on an mbarrier that
// nothing arrives on; when the wait gives up it raises the flag exactly as a
// step kernel whose staged rows never landed does.
__global__ void k_wait_selftest(int* __restrict__ err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0, limit)) atomicOr(err, 1);
}

extern "C" {

int lbm_selftest_wait_timeout(lbm_handle* h) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  k_wait_selftest<<<1, 32, 0, h->stream>>>(h->derr, 1LL << 12);
  CUDA_TRY(h, cudaGetLastError());
  return LBM_OK;
}

int64_t lbm_time(const lbm_handle* h) { return h ? h->t : -1; }

int64_t lbm_device_bytes(const lbm_handle* h) { return h ? h->bytes : 0; }

void lbm_destroy(lbm_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  while (!h->blocks.empty()) dev_free(h, h->blocks.back().first);
  delete h;
}

const char* lbm_last_error(const lbm_handle* h) { return h ? h->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Population / history export that allocates no device memory.
//
// lbm_fields stages each exported plane in a device buffer that the handle
// creates on first use.  Some callers cannot let the library allocate at
// that point: applications that reserve all device memory up front and
// forbid later allocations, and callers running with the device already
// full.  lbm_fields_noalloc exports the same planes through a fixed staging
// array compiled into the library instead.
//
// The array is a file-scope __device__ variable of NOALLOC_MAX_NODES
// doubles (8 MiB).  Every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current (the handle's device:
// a call made while another device is current is refused).  That first call
// should come before any stream capture begins.  The per-device address
// cache is atomic: host threads that make their first calls at the same
// time each look up the same address and store it, which is harmless.
//
// All calls share the one array, and it keeps whatever the last call left
// in it.  The export overwrites every element it later reads, so nothing
// needs clearing first.  Calls that run at the same time on the GPU (on
// different streams or handles) race on the array.
// ---------------------------------------------------------------------------
static constexpr long long NOALLOC_MAX_NODES = 1LL << 20;
static constexpr int NOALLOC_MAX_DEVICES = 64;
static __device__ __align__(256) double g_noalloc_stage[NOALLOC_MAX_NODES];
static std::atomic<double*> g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address per device ordinal

static int noalloc_stage_for_device(lbm_handle* h, double** out) {
  int dev = -1;
  CUDA_TRY(h, cudaGetDevice(&dev));
  if (dev != h->device)
    return fail(h, LBM_EINVAL, "lbm_fields_noalloc: device %d is current, but the handle lives on device %d", dev,
                h->device);
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(h, LBM_EINVAL, "device %d out of range", dev);
  double* a = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!a) {
    void* p = nullptr;
    CUDA_TRY(h, cudaGetSymbolAddress(&p, g_noalloc_stage));
    a = static_cast<double*>(p);
    g_noalloc_addr[dev].store(a, std::memory_order_release);
  }
  *out = a;
  return LBM_OK;
}

template <class C>
static int do_fields_noalloc(lbm_handle* h, int which, double* out, double* stage) {
  using T = typename C::value_t;
  const Phys<T> P = make_phys<T>(h);
  const T* src = nullptr;
  int NP = 0;
  double add0 = 0.0;
  if constexpr (C::dev) {  // decoded straight into the staging array
    if (which == LBM_F_POP || which == LBM_G_POP)
      return export_pulled<C>(h, which == LBM_F_POP ? 0 : 1, out, Region{0, 0, h->nx, h->ny}, stage);
  }
  if (which == LBM_F_POP || which == LBM_G_POP) {
    const int s = which == LBM_F_POP ? 0 : 1;
    T* spare = (T*)h->pops[s][1 - h->cur];  // allocated by lbm_create
    CUDA_TRY(h, launch_pull<T>(P, (const T*)h->pops[s][h->cur], spare, h->stream));
    src = spare;
    NP = 9;
    add0 = s == 1 ? h->prm.rho0 : 0.0;
  } else {
    src = (const T*)h->hist;
    NP = 5;
  }
  const long long N = (long long)h->nx * h->ny;
  for (int k = 0; k < NP; ++k) {
    CUDA_TRY(h, launch_export<T>(P, src, NP, k, stage, k == 0 ? add0 : 0.0, 0, 0, h->nx, h->ny, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(out + k * N, stage, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

extern "C" int lbm_fields_noalloc(lbm_handle* h, int32_t which, double* out) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!out) return fail(h, LBM_EINVAL, "out is NULL");
  if (which != LBM_F_POP && which != LBM_G_POP && which != LBM_HIST)
    return fail(h, LBM_EINVAL, "lbm_fields_noalloc exports only LBM_F_POP, LBM_G_POP and LBM_HIST (got %d)", which);
  const long long N = (long long)h->nx * h->ny;
  if (N > NOALLOC_MAX_NODES)
    return fail(h, LBM_EINVAL, "lbm_fields_noalloc handles at most %lld nodes; this grid has %lld (use lbm_fields)",
                NOALLOC_MAX_NODES, N);
  double* stage = nullptr;
  int rc = noalloc_stage_for_device(h, &stage);
  if (rc) return rc;
  PFLBM_DISPATCH(h, do_fields_noalloc, h, which, out, stage);
}

// ---------------------------------------------------------------------------
// Snapshots and the discrete adjoint of the Allen-Cahn step
// (pflbm_adjoint.cuh).  A snapshot is the f* set, the g* set and the five
// history planes, byte for byte in the handle's layout.
// ---------------------------------------------------------------------------
static long long state_bytes(const lbm_handle* h) {
  return 2 * h->pop_bytes + 5LL * h->plane * (long long)h->esize;
}

static int ensure_adjoint(lbm_handle* h) {
  if (h->have_adj) return LBM_OK;
  const size_t pl = (size_t)h->plane * h->esize;
  void* planes = dev_alloc(h, 51 * pl);  // lf 9, lg 9, lh 5, lp9 9, lfp 9, lgp 9, phi 1
  void* lext = dev_alloc(h, (size_t)(h->nx + 2) * (h->ny + 2) * h->esize);
  const long long nblocks = (long long)((h->nx + ADJ_THREADS - 1) / ADJ_THREADS) * h->ny;
  double* gpart = (double*)dev_alloc(h, (size_t)(2 * nblocks) * sizeof(double));
  double* gacc = (double*)dev_alloc(h, 2 * sizeof(double));
  if (!planes || !lext || !gpart || !gacc) {
    for (void* q : {planes, lext, (void*)gpart, (void*)gacc}) dev_free(h, q);
    return fail(h, LBM_ENOMEM, "adjoint work space (%zu bytes of planes)", 51 * pl);
  }
  unsigned char* b = static_cast<unsigned char*>(planes);
  h->adj.lf = b;
  h->adj.lg = b + 9 * pl;
  h->adj.lh = b + 18 * pl;
  h->adj.lp9 = b + 23 * pl;
  h->adj.lfp = b + 32 * pl;
  h->adj.lgp = b + 41 * pl;
  h->adj.phi = b + 50 * pl;
  h->adj.lext = lext;
  h->adj.gpart = gpart;
  h->gacc = gacc;
  CUDA_TRY(h, cudaMemsetAsync(planes, 0, 51 * pl, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(gacc, 0, 2 * sizeof(double), h->stream));
  h->have_adj = true;
  return LBM_OK;
}

static int adjoint_supported(lbm_handle* h) {
  if (h->dobs) return fail(h, LBM_EUNSUPPORTED, "the adjoint does not cover solid obstacles");
  if (h->slab) return fail(h, LBM_EUNSUPPORTED, "the adjoint does not cover y-slabs");
  if (h->prm.phase_model != LBM_AC)
    return fail(h, LBM_EUNSUPPORTED, "the adjoint covers the Allen-Cahn phase field only");
  if (h->prec != LBM_FP64 && h->prec != LBM_FP32)
    return fail(h, LBM_EUNSUPPORTED, "the adjoint needs FP64 or FP32 population storage");
  return LBM_OK;
}

template <typename T>
static int do_adjoint_seed(lbm_handle* h, const double* djdphi) {
  const Phys<T> P = make_phys<T>(h);
  int rc = ensure_stage(h, 1);
  if (rc) return rc;
  const long long N = (long long)h->nx * h->ny;
  CUDA_TRY(h, cudaMemcpyAsync(h->dstage, djdphi, N * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, launch_adjoint_seed<T>(P, h->dstage, h->adj, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->gacc, 0, 2 * sizeof(double), h->stream));
  return LBM_OK;
}

template <typename T>
static int do_adjoint_step(lbm_handle* h, const void* state) {
  const Phys<T> P = make_phys<T>(h);
  CUDA_TRY(h, launch_adjoint_step<T>(P, state, h->pop_bytes, h->adj, h->gacc, false, h->stream));
  return LBM_OK;
}

template <typename T>
static int do_adjoint_init(lbm_handle* h, const void* state0, double* out) {
  const Phys<T> P = make_phys<T>(h);
  int rc = ensure_stage(h, 1);
  if (rc) return rc;
  CUDA_TRY(h, launch_adjoint_step<T>(P, state0, h->pop_bytes, h->adj, h->gacc, true, h->stream));
  CUDA_TRY(h, launch_adjoint_init<T>(P, h->adj, h->dstage, h->stream));
  const long long N = (long long)h->nx * h->ny;
  CUDA_TRY(h, cudaMemcpyAsync(out, h->dstage, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

extern "C" {

int64_t lbm_state_bytes(const lbm_handle* h) { return h ? state_bytes(h) : 0; }

int lbm_snapshot(lbm_handle* h, void* dst) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!dst) return fail(h, LBM_EINVAL, "dst is NULL");
  unsigned char* d = static_cast<unsigned char*>(dst);
  CUDA_TRY(h, cudaMemcpyAsync(d, h->pops[0][h->cur], h->pop_bytes, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(d + h->pop_bytes, h->pops[1][h->cur], h->pop_bytes, cudaMemcpyDeviceToDevice,
                              h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(d + 2 * h->pop_bytes, h->hist, 5 * h->plane * h->esize, cudaMemcpyDeviceToDevice,
                              h->stream));
  return LBM_OK;
}

int lbm_restore(lbm_handle* h, const void* src, int64_t t) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!src || t < 0) return fail(h, LBM_EINVAL, "src is NULL or t < 0");
  const unsigned char* s = static_cast<const unsigned char*>(src);
  CUDA_TRY(h, cudaMemcpyAsync(h->pops[0][h->cur], s, h->pop_bytes, cudaMemcpyDeviceToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->pops[1][h->cur], s + h->pop_bytes, h->pop_bytes, cudaMemcpyDeviceToDevice,
                              h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->hist, s + 2 * h->pop_bytes, 5 * h->plane * h->esize, cudaMemcpyDeviceToDevice,
                              h->stream));
  h->t = t;
  return LBM_OK;
}

int lbm_adjoint_seed(lbm_handle* h, const double* dJ_dphi) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!dJ_dphi) return fail(h, LBM_EINVAL, "dJ_dphi is NULL");
  int rc = adjoint_supported(h);
  if (!rc) rc = ensure_adjoint(h);
  if (rc) return rc;
  return h->prec == LBM_FP64 ? do_adjoint_seed<double>(h, dJ_dphi) : do_adjoint_seed<float>(h, dJ_dphi);
}

int lbm_adjoint_step(lbm_handle* h, const void* state) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!state) return fail(h, LBM_EINVAL, "state is NULL");
  int rc = adjoint_supported(h);
  if (rc) return rc;
  if (!h->have_adj) return fail(h, LBM_EINVAL, "lbm_adjoint_seed has not been called");
  return h->prec == LBM_FP64 ? do_adjoint_step<double>(h, state) : do_adjoint_step<float>(h, state);
}

int lbm_adjoint_init(lbm_handle* h, const void* state0, double* dJ_dphi0) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!state0 || !dJ_dphi0) return fail(h, LBM_EINVAL, "state0 or dJ_dphi0 is NULL");
  int rc = adjoint_supported(h);
  if (rc) return rc;
  if (!h->have_adj) return fail(h, LBM_EINVAL, "lbm_adjoint_seed has not been called");
  if (!h->init_u_zero)
    return fail(h, LBM_EUNSUPPORTED, "lbm_adjoint_init differentiates lbm_init_fields with u = 0 only");
  return h->prec == LBM_FP64 ? do_adjoint_init<double>(h, state0, dJ_dphi0)
                             : do_adjoint_init<float>(h, state0, dJ_dphi0);
}

int lbm_adjoint_gravity(lbm_handle* h, double* dJ_dG) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!dJ_dG) return fail(h, LBM_EINVAL, "dJ_dG is NULL");
  if (!h->have_adj) return fail(h, LBM_EINVAL, "lbm_adjoint_seed has not been called");
  CUDA_TRY(h, cudaMemcpyAsync(dJ_dG, h->gacc, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return check_device_flag(h);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// y-slab decomposition of one grid over several devices or handles.
//
// A slab owns the global rows [y_lo, y_lo + ny_own).  It is an ordinary
// handle over ny_own + ghost_lo + ghost_hi local rows: LBM_SLAB_GHOST ghost
// rows below and above its own rows, except on a side that is a global wall
// (the wall is then the slab's own).  The step kernels run unchanged over the
// local rows.  A node's update reads populations at most three rows away
// (Cahn-Hilliard: phi two rows away feeds mu_phi one row away; Allen-Cahn:
// two), and the macroscopic pass of the diagnostics one row more, so once
// the ghost rows hold the neighbours' post-collision populations, every own
// row advances exactly as in the undivided grid.  The ghost rows themselves
// are then stale (their update saw the local grid's far edge, a wall or the
// periodic wrap), and the next halo exchange overwrites them.
//
// Exchange per step and side: the LBM_SLAB_GHOST own rows next to the side,
// of the f set and of the g set, post-collision (one contiguous block each:
// rows are row-interleaved, all nine planes of a row adjacent).  lbm_slab_pack
// copies them out, lbm_slab_unpack writes a neighbour's message into the
// ghost rows.  The history and phi(t-1) are per node and never exchanged.
// ---------------------------------------------------------------------------
static long long pop_row_bytes_of(const lbm_handle* h) { return h->pop_bytes / h->ny; }

extern "C" {

int lbm_create_slab(const lbm_params* global, int32_t y_lo, int32_t ny_own, void* stream,
                    const lbm_allocator* alloc, lbm_handle** out) {
  if (!out) return fail(nullptr, LBM_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(global);
  if (rc) return rc;
  const bool wy = global->bc[LBM_BOTTOM] == LBM_WALL;
  if (ny_own < LBM_SLAB_GHOST || y_lo < 0 || (long long)y_lo + ny_own > global->ny)
    return fail(nullptr, LBM_EINVAL, "slab rows [%d, %d) must lie in [0, %d) and number at least %d", y_lo,
                y_lo + ny_own, global->ny, LBM_SLAB_GHOST);
  if (ny_own == global->ny) return fail(nullptr, LBM_EINVAL, "a slab over the whole grid: use lbm_create");
  lbm_params loc = *global;
  const int glo = (wy && y_lo == 0) ? 0 : LBM_SLAB_GHOST;
  const int ghi = (wy && y_lo + ny_own == global->ny) ? 0 : LBM_SLAB_GHOST;
  loc.ny = ny_own + glo + ghi;
  rc = validate(&loc);
  if (rc) return rc;
  lbm_handle* h = nullptr;
  rc = create_impl(&loc, stream, alloc, &h);
  if (rc) return rc;
  h->slab = true;
  h->slab_y0 = y_lo;
  h->slab_own = ny_own;
  h->ghost_lo = glo;
  h->ghost_hi = ghi;
  *out = h;
  return LBM_OK;
}

int lbm_slab_info(const lbm_handle* h, int32_t info[4]) {
  if (!h || !info) return fail(nullptr, LBM_EINVAL, "handle or info is NULL");
  info[0] = h->slab ? h->slab_y0 : 0;
  info[1] = h->slab ? h->slab_own : h->ny;
  info[2] = h->ghost_lo;
  info[3] = h->ghost_hi;
  return LBM_OK;
}

int64_t lbm_slab_halo_bytes(const lbm_handle* h) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  return 2LL * LBM_SLAB_GHOST * pop_row_bytes_of(h);
}

// rows [first, first + LBM_SLAB_GHOST) of the current f and g sets <-> buf
static int slab_copy(lbm_handle* h, int side, void* buf, bool pack) {
  if (!h) return fail(nullptr, LBM_EINVAL, "handle is NULL");
  if (!buf) return fail(h, LBM_EINVAL, "buffer is NULL");
  if (!h->slab) return fail(h, LBM_EINVAL, "not a y-slab (lbm_create_slab)");
  if (side != LBM_BOTTOM && side != LBM_TOP) return fail(h, LBM_EINVAL, "side %d: LBM_BOTTOM or LBM_TOP", side);
  const int ghosts = side == LBM_BOTTOM ? h->ghost_lo : h->ghost_hi;
  if (!ghosts) return fail(h, LBM_EINVAL, "side %d of this slab is a global wall: nothing to exchange", side);
  int first;
  if (pack) first = side == LBM_BOTTOM ? h->ghost_lo : h->ghost_lo + h->slab_own - LBM_SLAB_GHOST;
  else first = side == LBM_BOTTOM ? 0 : h->ghost_lo + h->slab_own;
  const long long rb = pop_row_bytes_of(h), bytes = LBM_SLAB_GHOST * rb;
  for (int set = 0; set < 2; ++set) {
    unsigned char* rows = static_cast<unsigned char*>(h->pops[set][h->cur]) + first * rb;
    unsigned char* msg = static_cast<unsigned char*>(buf) + set * bytes;
    if (pack) CUDA_TRY(h, cudaMemcpyAsync(msg, rows, bytes, cudaMemcpyDeviceToDevice, h->stream));
    else CUDA_TRY(h, cudaMemcpyAsync(rows, msg, bytes, cudaMemcpyDeviceToDevice, h->stream));
  }
  return LBM_OK;
}

int lbm_slab_pack(lbm_handle* h, int32_t side, void* dst) { return slab_copy(h, side, dst, true); }

int lbm_slab_unpack(lbm_handle* h, int32_t side, const void* src) {
  return slab_copy(h, side, const_cast<void*>(src), false);
}

}  // extern "C"
