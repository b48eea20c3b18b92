/*
 * pflbm.h -- C-ABI of the GB300 phase-field lattice Boltzmann library.
 *
 * The library advances the consistent and conservative phase-field lattice
 * Boltzmann method of Zhan, Chai & Shi (arXiv:2111.00847) on one CUDA
 * device.  One time step t -> t+1 over the whole grid is one launch of a
 * fused kernel that pulls the D2Q9 populations f_i (phase field) and g_i
 * (hydrodynamics), evaluates phi = sum_i f_i on a halo ring, the isotropic
 * stencils of Eqs. (C.9)-(C.10), the chemical potential (Eq. (5)), the
 * Allen-Cahn (Eq. (7)) or Cahn-Hilliard (Eq. (6)) diffusion flux, the
 * consistent mass flux m^{phi C} (Eq. (15)), velocity (Eq. (22b)) and pressure
 * (Eq. (39), second way of Remark 1), and both MRT collisions (Eqs. (17),
 * (40)) with the moment vectors of Eqs. (C.2)-(C.4), then stores the
 * post-collision populations for the next pull.
 *
 * Conventions shared by every entry point
 *  - Grid: nx x ny nodes, node (i, j) at (i + 1/2, j + 1/2); host fields are
 *    row-major double arrays [ny][nx] (x fastest).  Population arrays are
 *    [9][ny][nx] in the D2Q9 order c_0 = (0,0), c_1 = (1,0), c_2 = (0,1),
 *    c_3 = (-1,0), c_4 = (0,-1), c_5 = (1,1), c_6 = (-1,1), c_7 = (-1,-1),
 *    c_8 = (1,-1) (the order fixed by the matrix of Eq. (C.1)).
 *  - Boundaries: each side is periodic or a half-way bounce-back wall (no
 *    slip for g, no flux for f, Sec. 4) with the wetting condition of
 *    Eqs. (49)-(50) at the contact angle of that side.
 *  - Return codes: LBM_OK (0) or a negative LBM_E* code; nothing aborts and
 *    no entry point throws.  lbm_last_error() describes the last failure.
 *  - Threading: a handle is not re-entrant; calls on one handle must not
 *    overlap.  Different handles are independent.
 *  - Streams: all device work of a handle runs on the CUDA stream given to
 *    lbm_create (NULL: the legacy default stream).  lbm_step is asynchronous
 *    unless diagnostics are due; lbm_init_fields, lbm_fields and
 *    lbm_set_fields synchronise the stream before returning.
 */
#ifndef PFLBM_H
#define PFLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 1
#define LBM_NDIAG 8

/* return codes */
enum {
    LBM_OK = 0,
    LBM_EINVAL = -1,       /* bad argument or parameter (message in lbm_last_error) */
    LBM_ENOMEM = -2,       /* device or host allocation failed */
    LBM_ECUDA = -3,        /* a CUDA call failed (message names the call) */
    LBM_EUNSTABLE = -4,    /* diagnostics found a non-finite value or |u| > 0.4 */
    LBM_EUNSUPPORTED = -5  /* valid but not implemented in this build */
};

/* lbm_params.precision: storage and arithmetic type of the populations.
 *   FP64, FP32: populations, history and arithmetic in that type.
 *   FP16_DEV, BF16_DEV: FP32 arithmetic and history; per population set and
 *     node the rest population (f_0, g_0) is stored in FP32 and the eight
 *     moving ones as 16-bit deviations s (q_i - r_i q_0) from the share the
 *     node holds at rest (r_i = 9 w_i eta / (9 - 5 eta) for the Allen-Cahn
 *     f, 0 for the Cahn-Hilliard f, -9 w_i / 5 for g; s a power of two).
 *     The stored f_0 is solved so that a node's nine decoded f sum to its
 *     phi, so total phi is conserved independently of the 16-bit rounding.
 *     FP16_DEV takes s = 2^(13 - ceil(log2 m)) with m = max(|phi_A|, |phi_B|)
 *     for f and max(rho_A, rho_B) for g, and needs both m in (2^-12, 2^28]
 *     (else LBM_EINVAL) so that s and 1/s are exact FP16 values; BF16_DEV
 *     takes s = 1.  An extension beyond the paper, which computes in double
 *     precision. */
enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_DEV = 2, LBM_BF16_DEV = 3 };
/* lbm_params.phase_model: D(phi) of Eq. (1) */
enum { LBM_AC = 0 /* Eq. (7), conservative Allen-Cahn */, LBM_CH = 1 /* Eq. (6), Cahn-Hilliard */ };
/* lbm_params.flux_model (Sec. 4): present = consistent flux rho u + m^{phi C};
 * original = m = rho u */
enum { LBM_PRESENT = 0, LBM_ORIGINAL = 1, LBM_CORRECTED = 2 };
/* lbm_params.visc_law: Eq. (11) (linear dynamic viscosity) or Eq. (12) */
enum { LBM_LINEAR_MU = 0, LBM_INVERSE_NU = 1 };
/* lbm_params.gravity_mode: body force G added to F = mu_phi grad phi + G
 *   CONST: G = (gx, gy)                         (Sec. 4.2)
 *   RHO:   G = rho (gx, gy)                     (Sec. 4.5)
 *   RHO_MINUS_MEAN: G = (rho - (rhoA+rhoB)/2) (gx, gy)   (Sec. 4.4) */
enum { LBM_G_CONST = 0, LBM_G_RHO = 1, LBM_G_RHO_MINUS_MEAN = 2 };
/* lbm_params.bc[side] */
enum { LBM_PERIODIC = 0, LBM_WALL = 1 };
enum { LBM_LEFT = 0, LBM_RIGHT = 1, LBM_BOTTOM = 2, LBM_TOP = 3 };
/* lbm_params.flags */
enum { LBM_FLAG_NO_TMA = 1 };
/* ghost rows on each exchanging side of a y-slab (lbm_create_slab) */
enum { LBM_SLAB_GHOST = 4 };
/* lbm_fields / lbm_set_fields selector */
enum {
    LBM_PHI = 0,   /* order parameter phi = sum_i f_i          [ny][nx]    */
    LBM_UX = 1,    /* velocity u, Eq. (22b)                    [ny][nx]    */
    LBM_UY = 2,    /* velocity v                               [ny][nx]    */
    LBM_P = 3,     /* pressure p, Eq. (39)                     [ny][nx]    */
    LBM_RHO = 4,   /* density rho(phi), Eq. (10)               [ny][nx]    */
    LBM_F_POP = 5, /* f_i(x, t) as seen by each node           [9][ny][nx] */
    LBM_G_POP = 6, /* g_i(x, t) as seen by each node           [9][ny][nx] */
    LBM_HIST = 7,  /* chi(t-1): phi u, phi v, u.m, u mx - v my, u my + v mx  [5][ny][nx] */
    LBM_DIAG = 8,  /* last diagnostics record                  [LBM_NDIAG] */
    LBM_MU = 9,    /* chemical potential mu_phi, Eq. (5)       [ny][nx]    */
    LBM_MCX = 10,  /* m^{phi C} x, Eq. (15)                    [ny][nx]    */
    LBM_MCY = 11   /* m^{phi C} y                              [ny][nx]    */
};

/*
 * Problem parameters, in the terms the paper states the problem (lattice
 * units, dx = dt = 1, c_s^2 = 1/3).
 *  version      must be LBM_ABI_VERSION
 *  nx, ny       grid size, each >= 3, nx*ny < 2^31
 *  phiA > phiB  order parameter of the two bulk phases (AC: 1, 0; CH: 1, -1)
 *  rhoA, rhoB   densities; rho(phi) linear, Eq. (10)
 *  muA, muB     dynamic viscosities; nu = mu / rho
 *  mobility     M_phi
 *  width        interface width W;  sigma  surface tension (Eq. (3) gives beta, k)
 *  eta          adjustable constant of Eqs. (C.3)-(C.4); 1 is the paper's value
 *  gx, gy       gravity / body-force vector, see gravity_mode
 *  rho0         constant of alpha_0 in Eq. (19)
 *  theta_deg    contact angle of each side (used where bc == LBM_WALL)
 *  s_f, s_g     MRT relaxation rates; NaN selects the default of Sec. 4:
 *               s_f^3 = s_f^5 = 1/(M_phi/(eta c_s^2) + 1/2),
 *               s_g^7 = s_g^8 = 1/(nu(phi)/c_s^2 + 1/2) per node, others 1
 *  diag_every   if > 0, lbm_step computes the diagnostics every diag_every
 *               steps (and then synchronises) and fails with LBM_EUNSTABLE
 *               on a non-finite value or |u| > 0.4
 *  flags        LBM_FLAG_NO_TMA: step with the register-pipelined kernel
 *               instead of the TMA-staged ones (Allen-Cahn and
 *               Cahn-Hilliard; same arithmetic, for A/B comparison);
 *               0 otherwise.  Grids under 16 columns always use the
 *               register-pipelined kernel.
 *  n_delta      regularisation of the interface normal of Eq. (8),
 *               n = grad phi / (|grad phi|^4 + delta^4)^(1/4) with
 *               delta = n_delta (phiA - phiB) / W (the paper's grad phi /
 *               |grad phi| is undefined where grad phi = 0); 0 selects the
 *               default 5e-3, which keeps the step a smooth, well-conditioned
 *               function of phi (round-off-level gradients in the bulk cannot
 *               steer the sharpening flux; gradients through long unstable
 *               runs exist).  It weakens the sharpening in the far interface
 *               tails, phi (1 - phi) below about n_delta / 4, which flows with
 *               a large viscosity ratio feel (the layered channel of Sec. 4.2
 *               needs 1e-5); small values make rounding differences grow
 *               quickly on rough or unstable flows.  Must lie in [0, 1).
 */
typedef struct lbm_params {
    int32_t version, nx, ny, precision;
    int32_t phase_model, flux_model, visc_law, gravity_mode;
    int32_t bc[4];
    int32_t diag_every, flags;
    double phiA, phiB, rhoA, rhoB, muA, muB;
    double mobility, width, sigma, eta;
    double gx, gy, rho0;
    double theta_deg[4];
    double s_f[9], s_g[9];
    double n_delta;
} lbm_params;

typedef struct lbm_handle lbm_handle;

/*
 * Optional device-memory provider.  alloc(bytes, stream, ctx) returns device
 * memory of at least `bytes` bytes aligned to 256 bytes, or NULL on failure;
 * free(ptr, stream, ctx) releases it.  The Python binding passes PyTorch's
 * caching allocator here.  NULL: the library calls cudaMalloc / cudaFree.
 */
typedef struct lbm_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, void *stream, void *ctx);
    void *ctx;
} lbm_allocator;

/*
 * Create a simulation on the current CUDA device.
 *  params  validated here (LBM_EINVAL with a message on any bad field;
 *          LBM_EUNSUPPORTED for flux_model == LBM_CORRECTED)
 *  stream  cudaStream_t to run on, or NULL
 *  alloc   device-memory provider or NULL
 *  out     receives the handle (NULL on failure)
 * Device memory owned by the handle: 2 x 18 population planes (16-bit
 * deviation storage: 2 x 2 FP32 + 2 x 16 16-bit planes), 5 history planes
 * and one phi plane of the arithmetic type, plus work planes created on
 * first use by lbm_fields / diagnostics.  With 16-bit storage,
 * lbm_init_fields and lbm_set_fields of populations also hold 9 (18 for
 * init) FP32 scratch planes for the duration of the call.  All of it is
 * released by lbm_destroy.
 */
int lbm_create(const lbm_params *params, void *stream, const lbm_allocator *alloc,
               lbm_handle **out);

/*
 * Set the state at t = 0 from host fields (row-major [ny][nx] doubles, read
 * only during the call; ux, uy, p may be NULL for zero).  Reading of the
 * paper (which states no initial populations): f = f^eq(phi, u),
 * g = g^eq(p, u) with m^{phi C} of phi, then the history is set to the
 * values the scheme computes at t = 0, so the first step's time derivatives
 * vanish.
 */
int lbm_init_fields(lbm_handle *h, const double *phi, const double *ux, const double *uy,
                    const double *p);

/* Advance nsteps (>= 0) time steps.  Asynchronous on the handle's stream
 * except at diagnostic points (diag_every > 0). */
int lbm_step(lbm_handle *h, int64_t nsteps);

/*
 * Copy a field at the current time to host memory `out` (layout per the
 * selector; doubles).  Macroscopic fields are recomputed from the current
 * populations by the step kernel's own formulas.  LBM_DIAG returns the
 * diagnostics at the current time (computed now): t, sum phi, D_u^rms,
 * S_m^rms (Eqs. (42)-(43), averaged over nodes not adjacent to a wall),
 * max |u|, count of non-finite nodes, number of averaged nodes, 0.
 * S_m^rms needs phi(t-1): it is exact at diagnostic points of lbm_step and
 * at t = 0; elsewhere it uses the last recorded phi(t-1).
 */
int lbm_fields(lbm_handle *h, int32_t which, double *out);

/* As lbm_fields, restricted to the node rectangle [x0, x0+w) x [y0, y0+hgt)
 * (out: [planes][hgt][w] doubles).  Lets a caller sample a grid too large to
 * copy whole.  A rectangle outside the grid: LBM_EINVAL.  LBM_DIAG ignores
 * the rectangle. */
int lbm_fields_region(lbm_handle *h, int32_t which, int32_t x0, int32_t y0, int32_t w, int32_t hgt,
                      double *out);

/*
 * Same result as lbm_fields for LBM_F_POP, LBM_G_POP or LBM_HIST, but with
 * no device allocation at any point (the paper has no counterpart: this is
 * a service of the library).  For callers that cannot let the library
 * allocate: applications that reserve all device memory up front, callers
 * whose device is full.
 * Planes are staged in one fixed 8 MiB array inside the library
 * (1,048,576 doubles), so grids above 1,048,576 nodes get LBM_EINVAL, as
 * do other selectors.  The handle's device (the one current at lbm_create)
 * must be current: otherwise LBM_EINVAL.  The first call on each device
 * looks up that array's address; make it before any stream capture starts.
 * The looked-up addresses are kept in an atomic per-device cache, so first
 * calls from several host threads at once are safe.  The array is shared
 * by all calls and keeps the last call's contents; calls that run on the GPU
 * at the same time race on it.  Synchronises the handle's stream.
 */
int lbm_fields_noalloc(lbm_handle *h, int32_t which, double *out);

/* Overwrite LBM_F_POP, LBM_G_POP or LBM_HIST (layouts as in lbm_fields) from
 * host doubles, e.g. to resume from a checkpoint.  Other selectors:
 * LBM_EINVAL. */
int lbm_set_fields(lbm_handle *h, int32_t which, const double *in);

/*
 * Solid obstacles inside the grid (the dam break over an obstacle, Sec. 4.5).
 *  solid  host [ny][nx] bytes, nonzero = solid node (read during the call);
 *         NULL or all zero removes the obstacles.
 * A solid node takes no part in the flow.  A link whose upstream node is
 * solid reflects like a wall link (half-way bounce-back, Sec. 4), so the
 * solid surface lies half-way between a solid node and its fluid neighbour.
 * The paper states the wetting condition for plane walls only (Eqs.
 * (49)-(50)); at a solid node the isotropic stencils see the neutral-wetting
 * value of phi (and of mu_phi for Cahn-Hilliard): the mean over its fluid
 * axis neighbours, or, with none, over its fluid diagonal neighbours.  Next
 * to a plane of solid nodes this is the 90-degree wall ghost (the mirror
 * value).  Every field of lbm_fields is zero at solid nodes; the
 * diagnostics sum over fluid nodes and average over fluid nodes without a
 * reflecting link.
 * Takes effect from the next call; call it before lbm_init_fields so that
 * the initial state holds no populations at solid nodes.  With obstacles a
 * step first forms phi (Cahn-Hilliard: and mu_phi) on a whole plane and
 * fills it at the solid nodes next to fluid, then runs the TMA step kernel
 * reading those planes (3 launches a step; 5 for Cahn-Hilliard; with
 * LBM_FLAG_NO_TMA or under 16 columns a one-thread-per-node update instead).
 * Device memory: a 2-byte link word per node, two work planes of the
 * arithmetic type and the list of solid nodes next to fluid.  The adjoint
 * entry points return LBM_EUNSUPPORTED while obstacles are set.
 */
int lbm_set_solid(lbm_handle *h, const uint8_t *solid);

/*
 * Self-test of the failure path (no counterpart in the paper).  Launches on
 * the handle's stream one wait, with the step kernels' bounded wait, on a
 * barrier that nothing arrives on; after about 4 ms it gives up and raises
 * the handle's device flag, as a step kernel does when its staged rows
 * never land.  The next call that synchronises (lbm_fields, diagnostics)
 * returns LBM_ECUDA with that message and clears the flag; the handle and
 * its state stay usable.  Returns LBM_OK once launched.
 */
int lbm_selftest_wait_timeout(lbm_handle *h);

/* Number of time steps taken since lbm_init_fields. */
int64_t lbm_time(const lbm_handle *h);

/* Bytes of device memory the handle holds now. */
int64_t lbm_device_bytes(const lbm_handle *h);

/* Free the handle and all device memory it owns (NULL is ignored). */
void lbm_destroy(lbm_handle *h);

/* Message of the last failure on h (or of the last lbm_create failure when
 * h is NULL).  Valid until the next call on the handle. */
const char *lbm_last_error(const lbm_handle *h);

/* ---- Snapshots and the discrete adjoint (an extension beyond the paper) ----
 *
 * The state after t steps is (f*, g*, chi): the post-collision populations
 * and the history of the explicit-Euler time derivatives (App. C).  A
 * snapshot holds it byte for byte: lbm_state_bytes(h) bytes of DEVICE
 * memory on the handle's device, written and read in order on the handle's
 * stream (the caller owns the memory; no synchronisation is implied).
 * lbm_restore also sets the step counter to t.  The diagnostics' phi(t-1)
 * is not part of the state. */
int64_t lbm_state_bytes(const lbm_handle *h);
int lbm_snapshot(lbm_handle *h, void *dst);
int lbm_restore(lbm_handle *h, const void *src, int64_t t);

/* Reverse mode of lbm_step for an objective J(phi_N) of the phase field
 * after N steps (Allen-Cahn model, FP64 or FP32 storage; otherwise
 * LBM_EUNSUPPORTED).  The handle keeps the adjoint lambda of the state.
 *   lbm_adjoint_seed(h, dJ_dphi)  host [ny][nx] doubles dJ/dphi_N:
 *       lambda := dJ/ds_N through phi_N = sum of the pulled f (Eq. (22a));
 *       zeroes the accumulated dJ/dG.
 *   lbm_adjoint_step(h, state)  state = device snapshot of s_t, the input of
 *       the step t -> t+1: lambda_{t+1} -> lambda_t, and adds the step's
 *       dJ/dG (G the body force of F = mu_phi grad phi + G, i.e. (gx, gy)
 *       scaled by the gravity mode).  Call for t = N-1 down to 0.
 *   lbm_adjoint_init(h, state0, dJ_dphi0)  state0 = device snapshot taken
 *       right after lbm_init_fields(phi0, NULL, NULL, p): writes dJ/dphi0 to
 *       host [ny][nx] doubles (LBM_EUNSUPPORTED if that init had a velocity)
 *       and adds the set-up's dJ/dG.
 *   lbm_adjoint_gravity(h, dJ_dG)  host double[2]: dJ/dgx, dJ/dgy so far.
 * The step is smooth except where the wetting root's discriminant is
 * clamped; there the clamp's derivative is taken as zero. */
int lbm_adjoint_seed(lbm_handle *h, const double *dJ_dphi);
int lbm_adjoint_step(lbm_handle *h, const void *state);
int lbm_adjoint_init(lbm_handle *h, const void *state0, double *dJ_dphi0);
int lbm_adjoint_gravity(lbm_handle *h, double *dJ_dG);

/*
 * y-slab decomposition: one grid divided into bands of rows, one handle per
 * band (on one device or on several), with a halo exchange between steps.
 * The paper calls its scheme fully parallel (Introduction): a node's update
 * reads only its neighbours (the streaming of Eqs. (17) and (40), the
 * stencils of Eqs. (C.9)-(C.10)), so a band advances exactly as the same
 * rows of the undivided grid once its neighbours' boundary rows are known.
 *
 * lbm_create_slab: a handle over the global rows [y_lo, y_lo + ny_own) of
 *   the grid `global` describes (ny_own >= LBM_SLAB_GHOST, and less than
 *   the whole grid).  Locally it holds ghost_lo + ny_own + ghost_hi rows:
 *   LBM_SLAB_GHOST ghost rows on each side that borders another slab (with
 *   periodic y, both sides), none on a side that is a global wall.  Every
 *   other call works on the local rows: lbm_init_fields, lbm_set_fields and
 *   lbm_fields take and give [local rows][nx] arrays (pass the global
 *   initial fields of rows y_lo - ghost_lo ... y_lo + ny_own + ghost_hi - 1,
 *   wrapped in a periodic y).  lbm_step advances one step per call
 *   (LBM_EINVAL for more): after each step, and after lbm_init_fields or
 *   lbm_set_fields, exchange the halos before the next step.  The
 *   diagnostics (lbm_fields LBM_DIAG, taken after the exchange; at
 *   diag_every the step records phi(t-1) for S_m but computes nothing)
 *   cover the own rows; slabs combine exactly by summing the
 *   sums and weighting the rms values with their n_avg.  Solid obstacles and
 *   the adjoint: LBM_EUNSUPPORTED.
 * lbm_slab_info: info = {y_lo, ny_own, ghost_lo, ghost_hi} ({0, ny, 0, 0}
 *   for an undivided handle).
 * lbm_slab_halo_bytes: bytes of one side's halo message (negative: error).
 * lbm_slab_pack: copy the message of `side` (LBM_BOTTOM or LBM_TOP) into
 *   dst, device memory of at least lbm_slab_halo_bytes bytes: the
 *   LBM_SLAB_GHOST own rows next to that side of the f set, then of the g
 *   set (post-collision populations, the library's storage layout).
 * lbm_slab_unpack: write the neighbour's message (its pack of the facing
 *   side: the upper neighbour's LBM_BOTTOM message into this slab's
 *   LBM_TOP side) into the ghost rows of `side`.
 *   Both are asynchronous copies on the handle's stream; order the
 *   transport (a peer copy, NCCL) after the pack and before the unpack.  A
 *   side that is a global wall: LBM_EINVAL.
 */
int lbm_create_slab(const lbm_params *global, int32_t y_lo, int32_t ny_own, void *cuda_stream,
                    const lbm_allocator *alloc, lbm_handle **out);
int lbm_slab_info(const lbm_handle *h, int32_t info[4]);
int64_t lbm_slab_halo_bytes(const lbm_handle *h);
int lbm_slab_pack(lbm_handle *h, int32_t side, void *dst);
int lbm_slab_unpack(lbm_handle *h, int32_t side, const void *src);

#ifdef __cplusplus
}
#endif

#endif /* PFLBM_H */
