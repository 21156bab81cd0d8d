/*
 * lbm.h - C ABI of the GB300 (sm_103a) thermocapillary phase-field lattice
 * Boltzmann library.
 *
 * The method is that of Holzer, Mitchell, Leonardi and Ruede, "Development of
 * a central-moment phase-field lattice Boltzmann model for thermocapillary
 * flows" (arXiv 2401.03041):
 *   - conservative Allen-Cahn phase-field LB for phi            (Sec. 2.2, Eq. lb_interface,
 *                                                                Eq. phasefieldforce)
 *   - D3Q27 central-moment hydrodynamic LB, velocity-based      (Sec. 2.2, Eq. for g^eq,
 *     formulation, surface-tension and Marangoni forcing          Eq. F_s, Eq. sigma(T))
 *   - energy equation as a D3Q7/15/19/27 passive-scalar LB      (Sec. 2.3, Eq. lb_thermal)
 *     or as RK2 / RK4 finite differences                        (Sec. 2.3, Eq. rk2, Eq. rk4)
 *   - pull "one step, two grid" stream-collide, sweep order     (Sec. 4.1, Alg. 1, Alg. 2)
 *
 * Conventions for every entry point:
 *   - Lattice units (dx = dt = 1).  Cell (i, j, k) has its centre at
 *     (i + 1/2, j + 1/2, k + 1/2): an n-cell axis spans [0, n].  x and y are
 *     periodic; z is periodic or bounded by two walls on the faces z = 0 and
 *     z = nz (lbm_params.walls_z).  Droplet centres, heat-source positions,
 *     the background-gradient origin and the diagnostics' first moments use
 *     these coordinates; heater patches use integer cell indices.
 *   - Field layout: [z][y][x], x fastest; multi-component fields are stored
 *     component-major ([comp][z][y][x]).  N = nx * ny * nz.
 *   - The library owns its state (PDF double buffers and auxiliary fields),
 *     either in a caller-provided device workspace or, if none is given, in
 *     memory it allocates itself.  The caller owns every other pointer.
 *   - Work is enqueued asynchronously on the CUDA stream given at creation;
 *     only calls that return host data (lbm_get_fields to host memory,
 *     lbm_get_pdfs, lbm_get_diagnostics, lbm_step_diagnostics) synchronise
 *     that stream.
 *   - Every call validates its arguments and returns an lbm_status; no call
 *     aborts the process.  A CUDA error is sticky on its domain: further
 *     calls on it return LBM_ERR_CUDA.  lbm_last_error() returns a message
 *     for the calling thread's most recent failure.
 *   - Not thread-safe per domain: one host thread at a time per domain.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_domain lbm_domain;   /* opaque, library-owned */

typedef enum {
  LBM_OK = 0,
  LBM_ERR_ARG = -1,          /* invalid argument (message in lbm_last_error) */
  LBM_ERR_CUDA = -2,         /* CUDA runtime error (sticky on the domain)   */
  LBM_ERR_OOM = -3,          /* device allocation failed / workspace too small */
  LBM_ERR_STATE = -4,        /* call out of order (e.g. step before init)   */
  LBM_ERR_NONFINITE = -5,    /* diagnostics found NaN/Inf in the state      */
  LBM_ERR_TIMEOUT = -6,      /* a bounded wait ran out                      */
  LBM_ERR_UNSUPPORTED = -7   /* valid request this build does not implement */
} lbm_status;

/* PDF storage precision.  FP64: stored and computed in double.  FP32: stored
 * and computed in float.  FP16_STORE: stored in IEEE half, computed in float.
 * FP32 and FP16 store the shifted values p_i - w_i * s (s = 1/2 for h, 0 for
 * g, T_ref for f).  Macroscopic reductions are always accumulated in FP64. */
typedef enum { LBM_FP64 = 0, LBM_FP32 = 1, LBM_FP16_STORE = 2 } lbm_precision;

/* Energy-equation solver (Sec. 2.3). */
typedef enum {
  LBM_TH_D3Q7 = 0, LBM_TH_D3Q15 = 1, LBM_TH_D3Q19 = 2, LBM_TH_D3Q27 = 3,
  LBM_TH_RK2 = 4, LBM_TH_RK4 = 5
} lbm_thermal;

/* Storage of the PDF sets.  LBM_LAYOUT_TWO_GRID: two sets, each step reads
 * one and writes the other (the pull scheme of Sec. 4.1, "one step, two
 * grids").  LBM_LAYOUT_AA: one set updated in place with the AA pattern
 * (alternating a step that gathers from the neighbours and scatters to them
 * with a step that gathers and scatters within the cell; Sec. 4.1 discusses
 * such single-grid schemes), about half the memory; each step first writes
 * a (phi, T) field of the level for the finite differences.  Same results
 * (in FP64 those of the generic two-grid kernel to rounding, 1e-12); the adjoint
 * needs LBM_LAYOUT_TWO_GRID. */
typedef enum { LBM_LAYOUT_TWO_GRID = 0, LBM_LAYOUT_AA = 1 } lbm_layout;

/* Model parameters (Sec. 2.1-2.3).  lbm_default_params() fills defaults. */
typedef struct {
  double nu_L, nu_H;       /* kinematic viscosity of the light (phi=0) / heavy (phi=1) phase;
                              tau(phi) = tau_L + phi (tau_H - tau_L), tau = nu / c_s^2 + 1/2 */
  double rho_L, rho_H;     /* densities of the light / heavy phase, rho(phi) = rho_L
                              + phi (rho_H - rho_L).  With rho_L != rho_H the pressure and
                              viscous correction forces F_p = -p* c_s^2 (rho_H - rho_L) grad phi
                              and F_mu = nu (rho_H - rho_L) [grad u + grad u^T] . grad phi act
                              (Sec. 2.2; strain from the non-equilibrium moments of g).  rho
                              also enters the heat capacity rho c_p of the energy equation
                              (see cp_L, cp_H).  The adjoint needs rho_L == rho_H. */
  double mobility;         /* Allen-Cahn mobility M; omega_phi = 1 / (1/2 + M / c_s^2) */
  double xi;               /* interface width */
  double sigma_ref, sigma_T, T_ref;  /* sigma(T) = sigma_ref + sigma_T (T - T_ref) */
  double alpha_L, alpha_H; /* thermal conductivity kappa of the light / heavy phase,
                              kappa(phi) = alpha_L + phi (alpha_H - alpha_L) (Sec. 2.3); the
                              diffusivity is alpha = kappa / C with C = rho(phi) c_p(phi) (equal
                              to kappa at the default rho = c_p = 1).  Eq. temperature:
                              dT/dt = -u.grad T_total + alpha lap T + (grad kappa / C)
                              . grad T_total + q_T.  LB: per-cell rate omega_T = 1 / (1/2 +
                              alpha / c_s^2), source (grad kappa / C) . G + alpha (C' / C)
                              grad phi . grad T; RK: the right-hand side as written.  The
                              adjoint needs a constant alpha (kappa and C uniform). */
  double gravity[3];       /* body-force acceleration g (F_b = rho g) */
  int32_t walls_z;         /* 1: no-slip walls at both z faces, else periodic in z */
  double T_bottom, T_top;  /* wall temperatures (walls_z == 1) */
  double grad_T[3];        /* imposed background gradient G: T_total = T + G.(x - x0) */
  double grad_T_origin[3]; /* x0 */
  double eps_n;            /* n = grad phi / (|grad phi| + eps_n) */
  double omega_high;       /* rate of central moments of order >= 3; this build requires 1 */
  int32_t rk_isotropic_fd; /* RK solvers: 0 = 7-point Laplacian and central gradient,
                              1 = isotropic D3Q27 operators */
  double T_bottom_amp;     /* bottom wall temperature T_bottom + T_bottom_amp cos(omega x), */
  int32_t T_bottom_waves;  /* omega = 2 pi T_bottom_waves / nx, x the cell centre (Sec. 3.1
                              planar heated channel); 0 = uniform T_bottom */
  double wall_u_bottom[2]; /* tangential (x, y) velocity of the bottom / top wall (walls_z == 1;  */
  double wall_u_top[2];    /* the sheared channel of Sec. 3.3): bounce-back adds the wall's
                              momentum 2 w_i (c_i . u_w) / c_s^2 to g (times phi to h), and
                              the thermal anti-bounce-back takes the even part of the
                              equilibrium at u_w; |u_w| < 0.3 */
  double theta_bottom;     /* contact angle (degrees, measured through phi = 1) at the bottom /   */
  double theta_top;        /* top wall, 0 < theta < 180 (Sec. 3.3 wetting condition): the ghost
                              phi beyond the wall solves (a - g) = -(4 / xi) cos(theta) w (1 - w),
                              w = (a + g) / 2, a the first fluid cell; 90 = neutral (mirror) */
  double cp_L, cp_H;       /* specific heat capacity of the light / heavy phase, c_p(phi) =
                              cp_L + phi (cp_H - cp_L) (Sec. 2.3); > 0, default 1 */
} lbm_params;

/* Gaussian laser heat source, Eq. HeatSource: q = Q exp(-2 r^2 / w^2) where
 * r^2 <= d^2 (d <= 0 or infinite: no cut-off). */
typedef struct { double x, y, z, Q, w, d; } lbm_heat_source;

/* Spherical droplet for initialisation: phi = 1/2 (1 + tanh(2 (R - r) / xi)),
 * velocity (ux, uy, uz) weighted by the droplet's own phi. */
typedef struct { double cx, cy, cz, R, ux, uy, uz; } lbm_droplet;

/* FP64 diagnostics of one time level (Sec. 3.4 centroid tracking). */
typedef struct {
  double mass;      /* sum phi */
  double heat;      /* sum T (the evolved field, without the background G term) */
  double kinetic;   /* 1/2 sum rho |u|^2 */
  double mx, my, mz;/* sum phi x, sum phi y, sum phi z (no periodic unwrapping) */
  int64_t level;    /* time level the values describe */
  int32_t nonfinite;/* 1 if any summand was NaN/Inf */
  int32_t pad_;
} lbm_diag;

#define LBM_FIELD_PHI 1u   /* phi              (1 component)  */
#define LBM_FIELD_U   2u   /* velocity u       (3 components) */
#define LBM_FIELD_P   4u   /* normalised pressure p* (1)      */
#define LBM_FIELD_T   8u   /* temperature T    (1)            */

#define LBM_MAX_SOURCES  64
#define LBM_MAX_PATCHES  64
#define LBM_MAX_DROPLETS 4096

/* Fill *p with the defaults (the 32^3 periodic droplet workload's values). */
void lbm_default_params(lbm_params* p);

/* Device workspace bytes a domain needs (PDF double buffers for h (q_phase),
 * g (27) and f, RK stage fields, reduction scratch).  0 for invalid input. */
size_t lbm_workspace_bytes(int nx, int ny, int nz, lbm_precision prec,
                           lbm_thermal thermal, int q_phase);

/* Create a domain of nx * ny * nz cells (each >= 1, ny <= 262140, nz <= 65535;
 * N < 2^40).
 *   q_phase:   15 (D3Q15) or 27 (D3Q27) for the phase-field PDFs h.
 *   stream:    a cudaStream_t (NULL = legacy default stream).
 *   workspace: device pointer of at least lbm_workspace_bytes(...) bytes,
 *              256-byte aligned, owned by the caller and kept alive until
 *              lbm_destroy_domain; NULL makes the library allocate it.
 * Errors: LBM_ERR_ARG (sizes, enums), LBM_ERR_OOM, LBM_ERR_CUDA. */
lbm_status lbm_create_domain(int nx, int ny, int nz, lbm_precision prec,
                             lbm_thermal thermal, int q_phase, void* stream,
                             void* workspace, size_t workspace_bytes,
                             lbm_domain** out);

/* lbm_workspace_bytes / lbm_create_domain with a choice of PDF layout
 * (lbm_layout; the functions above use LBM_LAYOUT_TWO_GRID).  The in-place
 * layout holds one PDF set plus a (phi, T) field: about half the bytes of
 * the two-grid layout.  Every other call works on either layout;
 * lbm_get_pdfs / lbm_set_pdfs exchange the same post-collision populations
 * p_i(x) whatever the layout, and saved states record it (a state loads only
 * into a domain of the same layout).  Errors as lbm_create_domain, and
 * LBM_ERR_ARG for an unknown layout (lbm_workspace_bytes_layout: 0). */
size_t lbm_workspace_bytes_layout(int nx, int ny, int nz, lbm_precision prec,
                                  lbm_thermal thermal, int q_phase, lbm_layout pdf_layout);
lbm_status lbm_create_domain_layout(int nx, int ny, int nz, lbm_precision prec,
                                    lbm_thermal thermal, int q_phase, lbm_layout pdf_layout,
                                    void* stream, void* workspace, size_t workspace_bytes,
                                    lbm_domain** out);

/* Synchronise the domain's stream and release everything the library owns. */
lbm_status lbm_destroy_domain(lbm_domain* dom);

/* Set the model parameters (Sec. 2.1-2.3).  Copied; takes effect for the
 * next launch.  LBM_ERR_ARG for non-physical values (nu <= 0, M <= 0,
 * xi <= 0, rho <= 0, alpha <= 0, non-finite); LBM_ERR_UNSUPPORTED for
 * omega_high != 1. */
lbm_status lbm_set_params(lbm_domain* dom, const lbm_params* p);

/* Replace the Gaussian heat sources (0 <= n <= LBM_MAX_SOURCES; Eq. HeatSource,
 * read as non-zero inside r <= d).  src is host memory, copied. */
lbm_status lbm_set_heat_sources(lbm_domain* dom, int n, const lbm_heat_source* src);

/* Replace the rectangular heater patches on layer z (0 <= n <= LBM_MAX_PATCHES):
 * patch k adds heat source density intensity[k] on the cells
 * x0[k] <= x < x0[k] + sx, y0[k] <= y < y0[k] + sy of layer z.  Host arrays, copied. */
lbm_status lbm_set_heater_patches(lbm_domain* dom, int z, int sx, int sy, int n,
                                  const int32_t* x0, const int32_t* y0,
                                  const double* intensity);

/* Add a caller-given heat-source density field to q_T (the source term of
 * the temperature equation, Sec. 2.3), on top of the Gaussian sources and the
 * heater patches.  q_dev is a dense [nz][ny][nx] array (x fastest) in device
 * memory of the current device, of type double (dtype LBM_FP64) or float
 * (LBM_FP32), aligned to its element size.  It is NOT copied: the caller owns
 * it and keeps it alive and unchanged while steps that read it are in flight
 * (every later lbm_step / lbm_step_diagnostics / lbm_adjoint_run reads it).
 * NULL removes the field.  The source does not depend on the state, so the
 * adjoint of the state is unchanged by it.
 * Errors: LBM_ERR_ARG for a bad dtype, a misaligned, host or other-device
 * pointer; a domain's sticky error is returned again. */
lbm_status lbm_set_heater_field(lbm_domain* dom, const void* q_dev, int dtype);

/* Initialise the state from n droplets (0 <= n <= LBM_MAX_DROPLETS, host
 * array): phi = max_k phi_k (periodic minimum-image distances), u = sum_k phi_k v_k,
 * T = linear conduction profile between the walls (walls_z) else 0;
 * h = h^eq(phi, u), g = g^eq(0, u), f = f^eq(T, u) (Sec. 2.2 equilibria).
 * These PDFs are treated as the post-collision values of level 0: the first
 * step streams them.  Resets the level counter to 0. */
lbm_status lbm_init_droplets(lbm_domain* dom, int n, const lbm_droplet* d);

/* Advance nsteps >= 0 time steps (Alg. 1 / Alg. 2 order: h, g, then f or the
 * RK stages), asynchronously on the domain's stream. */
lbm_status lbm_step(lbm_domain* dom, int nsteps);

/* Advance nsteps >= 1 steps and return the FP64 diagnostics of the time level
 * the last step consumed (accumulated inside that step's kernel, no extra
 * pass).  Synchronises.  LBM_ERR_NONFINITE if a NaN/Inf was met (the step is
 * still taken and *out still written). */
lbm_status lbm_step_diagnostics(lbm_domain* dom, int nsteps, lbm_diag* out);

/* Diagnostics of the current time level (one extra read-only pass).  Synchronises. */
lbm_status lbm_get_diagnostics(lbm_domain* dom, lbm_diag* out);

/* Macroscopic fields of the current time level (what the next step computes
 * from its pulled PDFs): the fields selected by mask (LBM_FIELD_*) are written
 * in the order phi, u (3), p*, T, each N values, as double (dtype 0) or float
 * (dtype 1).  dst is a device pointer if dst_on_device, else host memory
 * (then the call synchronises).  dst must hold count * N values. */
lbm_status lbm_get_fields(lbm_domain* dom, unsigned mask, void* dst,
                          int dst_on_device, int dtype);

/* Copy one PDF set of the current state to host memory as FP64, un-shifted:
 * which = 0 (h, q_phase values), 1 (g, 27), 2 (f, thermal Q; LB thermal only)
 * or 3 (T field, 1 value; RK thermal only).  dst holds Q * N doubles.  Synchronises. */
lbm_status lbm_get_pdfs(lbm_domain* dom, int which, double* dst_host);

/* Overwrite one PDF set of the current state from FP64 host values (layout as
 * lbm_get_pdfs; shifted and rounded to the storage precision). */
lbm_status lbm_set_pdfs(lbm_domain* dom, int which, const double* src_host);

/* Checkpoint / resume (the paper describes none; a utility of the library).
 * lbm_state_bytes: bytes of a saved state of this domain (a header naming
 * the domain's sizes, precision, stencils and time level; the current PDF set
 * in its stored form, ghost cells included; for the RK energy solvers the T
 * field); 0 for a null domain.
 * lbm_save_state: copies the current state to host memory (host_buf, at
 * least lbm_state_bytes bytes, owned by the caller).  Synchronises.
 * LBM_ERR_ARG (null or short buffer), LBM_ERR_STATE (not initialised).
 * lbm_load_state: restores a state saved from a domain of the same sizes,
 * precision, thermal solver and phase-field stencil, including its time
 * level; the next step continues exactly as the saved run would have.
 * Synchronises.  LBM_ERR_ARG if the buffer is not such a state. */
size_t lbm_state_bytes(lbm_domain* dom);
lbm_status lbm_save_state(lbm_domain* dom, void* host_buf, size_t bytes);
lbm_status lbm_load_state(lbm_domain* dom, const void* host_buf, size_t bytes);

/* Current time level (number of steps since lbm_init_droplets). */
lbm_status lbm_get_level(lbm_domain* dom, int64_t* level);

/* Wait for the domain's stream with a bounded host-side wait (event polling);
 * LBM_ERR_TIMEOUT if the work has not finished after timeout_ms. */
lbm_status lbm_synchronize(lbm_domain* dom, int timeout_ms);

/* Launch configuration of the domain's step kernel: info[0] = 0 for the
 * generic kernel, 1 for the bulk kernel (PDF boxes staged in shared memory by
 * tensor-TMA copies), 2 for the skewed kernel (the same staging, the two
 * threads of a cell one plane apart), 3 for the in-place layout on the
 * generic tiles, 4 for the in-place layout on the skewed kernel's tiles (all
 * parameters but a density ratio, which runs it on the generic tiles);
 * info[1..3] = grid x, y, z (tile counts and z-chunks); info[4] = planes per
 * CTA; info[5] = dynamic shared memory bytes.  info holds 6 int32 values.
 * The environment variable LBM_KERNEL=generic, read at creation, forces the
 * generic kernels (two-grid and in-place), LBM_KERNEL=bulk the bulk kernel;
 * LBM_ZCHUNK=<planes> sets the planes per CTA.
 * LBM_TEST_STALL=1, read at creation, tests failure detection: the bulk
 * kernel's first copy wait of every CTA then runs out (after about 2 s per
 * wait, no fault), the kernel raises the domain's error flag and returns, and
 * the next call that synchronises (lbm_synchronize, lbm_get_diagnostics, ...)
 * returns LBM_ERR_TIMEOUT, which then sticks to the domain. */
lbm_status lbm_kernel_info(lbm_domain* dom, int32_t* info);

/* Gradient of a droplet-capture objective with respect to the heater-patch
 * intensities, by the discrete adjoint of the time step.  The paper has no
 * adjoint: this is the exact transpose of the linearised FP64 step of
 * lbm_step (Sec. 2.2-2.3 model, Alg. 1 sweep order), for FP64 storage with
 * the energy equation as the thermal LB (D3Q7/15/19/27) or RK2 / RK4 (Eq.
 * rk2, Eq. rk4; the state then holds the T field), a uniform diffusivity,
 * equal densities, walls at rest with neutral wetting, the two-grid layout,
 * a whole lattice and nx * ny < 2^31 (else LBM_ERR_UNSUPPORTED).
 *   Starting from the current state (level n0), runs nsteps steps forward,
 *   keeping a copy of the state every ckpt_every steps, and evaluates
 *   J = |c - target|^2, c = (sum phi x, sum phi y, sum phi z) / sum phi at
 *   level n0 + nsteps (cell-centred coordinates, no periodic unwrapping).
 *   Then it runs the adjoint steps backwards, replaying each checkpoint
 *   segment forward to recover the states it needs, and accumulates
 *   dJ/dI_k (I_k = intensity of patch k of lbm_set_heater_patches).
 *   On return the domain holds the forward result (level n0 + nsteps), *J_out
 *   is J and dJdI_host[k] (host memory, one double per patch; may be NULL)
 *   the gradient.
 *   normal_cap <= 0: the exact discrete adjoint.  normal_cap > 0: the
 *   interface normal n = grad phi / (|grad phi| + eps_n) is differentiated
 *   only in cells where |4 phi (1 - phi) / xi| <= normal_cap |grad phi| (on
 *   the equilibrium tanh profile the two sides are equal) and held fixed
 *   elsewhere.  In far-field tails and at extrema of phi the exact derivative
 *   of n grows like 4 phi (1 - phi) / (xi |grad phi|) without bound; over long
 *   horizons (thousands of steps) the exact linearised step then amplifies
 *   round-off-level perturbations there that the step itself keeps bounded,
 *   and the exact gradient no longer describes finite changes of J.
 *   Synchronises.  Allocates its buffers for the duration of the call:
 *   nsteps / ckpt_every + 1 states (PDF set, and the T field with RK:
 *   checkpoints, final state), ckpt_every x 19 doubles per cell (the replayed
 *   steps' intermediates), 3 dense adjoint sets (q_phase + 27 + Q_f doubles
 *   per cell each, Q_f = 1 for RK) and with RK 13 doubles per cell for the
 *   stage reverse: LBM_ERR_OOM if they do not fit.
 * Errors: LBM_ERR_ARG (nsteps < 1, ckpt_every < 1, null target / J_out, NaN normal_cap),
 * LBM_ERR_STATE (not initialised, zero phi mass), LBM_ERR_UNSUPPORTED. */
lbm_status lbm_adjoint_run(lbm_domain* dom, int nsteps, int ckpt_every, const double* target,
                           double normal_cap, double* J_out, double* dJdI_host);

/* One adjoint step at the current state s: lam_out = (d Phi / d s)^T lam_in,
 * where Phi is one lbm_step.  lam_in and lam_out are host arrays of
 * (q_phase + 27 + Q_f) * N doubles in the order of lbm_get_pdfs (h, then g,
 * then f, each [direction][z][y][x]; with RK2 / RK4 the T field [z][y][x]
 * takes the place of f, Q_f = 1); normal_cap as in lbm_adjoint_run.
 * Same requirements as lbm_adjoint_run;
 * allocates its buffers for the call; synchronises.  (The building block of
 * lbm_adjoint_run, exposed for dot-product tests against the linearised step.) */
lbm_status lbm_adjoint_step(lbm_domain* dom, const double* lam_in_host, double* lam_out_host,
                            double normal_cap);

/* Step-kernel timing, a measurement aid (the paper has no counterpart).
 * After lbm_profile_steps(dom, 1) each launch of the step kernel by lbm_step /
 * lbm_step_diagnostics (the first LBM_MAX_PROFILED since the last read) is
 * bracketed by CUDA events recorded on the domain's stream; the ghost-fill
 * and RK-stage launches are not included.  lbm_profile_steps(dom, 0) stops
 * recording.  lbm_profile_read synchronises the stream, returns the summed
 * duration (ms) and the number of timed launches, and resets the count. */
#define LBM_MAX_PROFILED 4096
lbm_status lbm_profile_steps(lbm_domain* dom, int enable);
lbm_status lbm_profile_read(lbm_domain* dom, double* ms_total, int32_t* launches);

/* Halo exchange of a decomposition into x slabs (Sec. 4.3: each slab holds
 * its own columns plus halo columns that the neighbouring slabs refresh
 * after every step).  A slab is a domain of its own (periodic in x, so its
 * halo columns hold garbage after a step until they are refreshed); a step
 * produces correct values wherever the step's dependencies (2 cells for the
 * LB energy solvers, 5 for RK4) stay inside the slab.
 *   lbm_halo_bytes:    bytes of the buffer for `width` columns: the stored
 *                      populations of every PDF set direction (storage
 *                      type), [direction (h, then g, then f)][z][y][width],
 *                      then, 16-byte aligned, the RK temperature [z][y][width]
 *                      (compute type); 0 for width outside [1, nx].
 *   lbm_pack_halo_x:   copy columns [x0, x0 + width) of the current state
 *                      into dst_dev (device memory, lbm_halo_bytes bytes).
 *   lbm_unpack_halo_x: copy src_dev into columns [x0, x0 + width) of the
 *                      current state (and refresh the tiled kernels'
 *                      periodic ghost copies).
 * Both are enqueued on the domain's stream (no synchronisation); moving the
 * buffer between slabs (NCCL, peer copies, host staging) is the caller's.
 * Errors: LBM_ERR_ARG (columns outside the lattice, null or non-device
 * buffer), LBM_ERR_STATE (not initialised), LBM_ERR_UNSUPPORTED (in-place
 * layout). */
/* Declare the domain an x slab of a larger lattice: local column x is global
 * column (x + x_offset) mod nx_global for every position-dependent term
 * (heat sources, heater patches, the background gradient, the modulated
 * bottom wall, droplets of lbm_init_droplets, the first moments of
 * lbm_diag), so that a slab with halo columns computes exactly what the
 * whole lattice computes in its own columns.  (0, nx) restores a whole
 * lattice.  LBM_ERR_ARG for nx_global < nx; LBM_ERR_UNSUPPORTED for the
 * in-place layout; the adjoint rejects sub-domains. */
lbm_status lbm_set_subdomain(lbm_domain* dom, int x_offset, int nx_global);

size_t lbm_halo_bytes(lbm_domain* dom, int width);
lbm_status lbm_pack_halo_x(lbm_domain* dom, int x0, int width, void* dst_dev);
lbm_status lbm_unpack_halo_x(lbm_domain* dom, int x0, int width, const void* src_dev);

/* FP64 mass and first moments of a caller-owned device field, computed
 * without allocating any memory.  The paper has no counterpart: this is a
 * utility of the library (the phi mass and centroid moments of lbm_diag, for
 * a field that need not belong to a domain, e.g. a phi field already copied
 * out with lbm_get_fields).
 *   out_host[0] = sum psi, out_host[1..3] = sum psi (x + 1/2), sum psi
 *   (y + 1/2), sum psi (z + 1/2) over the [z][y][x] field (cell-centred
 *   coordinates), accumulated in FP64 in a fixed order (deterministic).
 *   field:  pointer to nx * ny * nz values, double (dtype 0) or float
 *           (dtype 1), in device (or managed) memory of the CURRENT device;
 *           a host pointer or memory of another device is rejected with
 *           LBM_ERR_ARG before anything is launched.  nz <=
 *           LBM_MOMENTS_MAX_PLANES and nx * ny < 2^31, else LBM_ERR_ARG
 *           (nothing is launched).
 *   stream: cudaStream_t of the current device (NULL = legacy default
 *           stream); a stream of another device is LBM_ERR_ARG.  Two kernels
 *           and a 32-byte copy are enqueued on it, then it is synchronised.
 *   out_host: 4 doubles of host memory.
 * Why it exists: every other call that needs scratch memory takes it from the
 * domain's workspace.  Callers that must not allocate device memory at call
 * time and hold no domain (a process under a hard device-memory budget, or
 * one whose device memory all belongs to its own pool allocator) can use this
 * one: its scratch is a fixed array compiled into the library, about 128 KB
 * ((LBM_MOMENTS_MAX_PLANES + 1) x 4 doubles), whose contents never need to
 * start at zero (every call writes each slot before reading it).
 * The first call on a device looks up that array's device address, with the
 * device current; make it before any stream capture on that device.  A
 * lookup that fails is reported (LBM_ERR_CUDA) and retried by the next call.  Calls
 * that overlap in time on one device (from several host threads, or on
 * streams without ordering between them) share the array and race: serialise
 * them.  Errors: LBM_ERR_ARG, LBM_ERR_CUDA. */
#define LBM_MOMENTS_MAX_PLANES 4096
lbm_status lbm_field_moments(const void* field, int dtype, int nx, int ny, int nz,
                             void* stream, double* out_host);

/* Message of the calling thread's most recent failed call ("" if none). */
const char* lbm_last_error(void);

/* Velocity set of stencil Q (7, 15, 19 or 27) in the library's direction order
 * (rest; +x,-x,+y,-y,+z,-z; twelve edges; eight corners; App. B classes):
 * c_out[3*i + a] = component a of c_i, w_out[i] = w_i.  Either pointer may be NULL. */
lbm_status lbm_stencil(int Q, int32_t* c_out, double* w_out);

/* Library version string. */
const char* lbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
