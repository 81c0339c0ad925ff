/*
 * lbnci.h -- C ABI of the GB300 (sm_103a) two-component colour-gradient lattice
 * Boltzmann solver with near-contact interactions (NCI).
 *
 * Method: Montessori, Tiribocchi, Bonaccorso, Lauricella, Succi, "Lattice Boltzmann
 * simulations capture the multiscale physics of soft flowing crystals",
 * arXiv:2003.11069, section "Materials and Methods":
 *   - two population sets f_i^k (k = 1, 2) evolving by Eq. (CGLBE), dt = 1;
 *   - collision Omega = Omega^(3)[Omega^(1) + Omega^(2)]: BGK relaxation, the
 *     surface-tension perturbation and recolouring with segregation beta;
 *   - order parameter psi = (rho1 - rho2)/(rho1 + rho2), normal n = -grad psi/|grad psi|;
 *   - NCI force F_rep = -A_h[h(x)] n delta_I, delta_I = |grad psi|/2, Eq. (near_c),
 *     with A_h = A for h <= h_min, A (h_min/h)^3 for h_min < h <= h_max, 0 beyond.
 * A uniform body force G drives the flow; G and F_rep enter through Guo forcing.
 * Every entry point runs its arithmetic in this library's CUDA kernels; there is
 * no CPU fallback. A missing or unusable GPU makes lb_create fail with LB_ECUDA.
 *
 * Conventions
 *   Site index     idx = x + nx*(y + ny*z), x fastest; nz = 1 on D2Q9.
 *   Boundaries     x is periodic. y (and z on D3Q27) is periodic, or bounded by
 *                  halfway bounce-back walls just below index 0 and just above
 *                  index n-1 when wall_y (wall_z) is set.
 *   Velocities     direction i = 0..Q-1 has c_i given by the base-3 digits of i
 *                  (x from the lowest digit, then y, then z), digit d mapping to
 *                  {0, +1, -1}[d]. Weights: D2Q9 4/9, 1/9, 1/36; D3Q27 8/27, 2/27,
 *                  1/54, 1/216 by |c_i|^2.
 *   Populations    f[k][i][idx], k = 0 for component 1 (the dispersed phase,
 *                  psi > 0) and 1 for component 2. The state between steps is the
 *                  post-collision population at its own site; a step first pulls
 *                  (streams), then collides.
 *   Vectors        [3][N] arrays (component-major), z component 0 on D2Q9.
 *   Host/device    arrays are host pointers when on_device == 0 and device pointers
 *                  (on the sim's device) when on_device == 1. All host arrays are
 *                  FP64 (int32 for hit maps) whatever the storage precision.
 *
 * Ownership: the sim owns the memory it allocates; a caller-provided workspace
 * (lb_config.workspace) stays the caller's and must outlive the sim. Caller arrays
 * are only read or written during the call (or, for on_device == 1, in stream order
 * on lb_config.stream).
 *
 * Errors: every call returns an lb_status and never aborts or traps. lb_step
 * reports launch failures at once; numerical blow-up (a non-finite or non-positive
 * density) is reported by the next lb_observables / lb_fields as LB_ENUMERIC.
 * lb_last_error() gives a one-line description of the last failure. A sim handle
 * must not be used from two host threads at once.
 */
#ifndef LBNCI_H
#define LBNCI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LB_OK = 0,
  LB_EINVAL = 1,       /* bad argument or configuration */
  LB_ENOMEM = 2,       /* device allocation failed or workspace too small */
  LB_ECUDA = 3,        /* CUDA runtime error (no device, launch failure, ...) */
  LB_ENUMERIC = 4,     /* non-finite or non-positive density detected */
  LB_EUNSUPPORTED = 5  /* valid request this build does not implement */
} lb_status;

typedef enum { LB_D2Q9 = 0, LB_D3Q27 = 1 } lb_lattice;

typedef enum {
  LB_FP64 = 0,    /* populations stored and computed in FP64 (parity path) */
  LB_FP32 = 1,    /* populations stored and computed in FP32 */
  LB_FP16DEV = 2  /* populations stored as FP16 deviations f_i - w_i rho_k from the
                     lattice-weight equilibrium at rest, with FP32 reference densities
                     rho_k per site; arithmetic in FP32 */
} lb_precision;

typedef enum {
  /* Guo forcing of the mixture with u = (j + F/2)/rho, F = G + F_rep (default) */
  LB_FORCE_GUO = 0,
  /* The paper's own insertion ("Materials and Methods", last paragraph): exact
   * difference method, the near-contact force acting on the dispersed phase only. The
   * relaxation uses u = j/rho; after recolouring component k gains
   * f_eq(rho_k, u + dU_k) - f_eq(rho_k, u), dU_k = F_k/rho_k, with F_1 = G rho_1/rho +
   * F_rep and F_2 = G rho_2/rho. Reported velocities are still (j + F/2)/rho. */
  LB_FORCE_EDM_DISPERSED = 1
} lb_forcing;

typedef struct {
  int lattice;          /* lb_lattice */
  int nx, ny, nz;       /* lattice size; nz = 1 for D2Q9 */
  int wall_y, wall_z;   /* 1 = halfway bounce-back walls on that axis, 0 = periodic */
  double tau;           /* BGK relaxation time, nu = (tau - 1/2)/3; tau > 1/2 */
  double A_s;           /* perturbation amplitude of each component; sigma = 4 A_s tau/9 */
  double beta;          /* recolouring segregation parameter, 0 <= beta <= 1 */
  double A_h;           /* NCI strength A (force per unit volume); 0 disables NCI */
  double h_min, h_max;  /* NCI cut-offs in lattice units, 0 < h_min <= h_max < 5 */
  double g_th;          /* interface threshold on |grad psi| for the NCI ray search */
  double force[3];      /* uniform body-force density G */
  int precision;        /* lb_precision */
  void* stream;         /* cudaStream_t for all work; NULL = the legacy default stream */
  void* workspace;      /* optional caller-owned device memory, 256-byte aligned */
  size_t workspace_bytes;
  int forcing;          /* lb_forcing: how G and F_rep enter the populations */
} lb_config;

typedef struct lb_sim lb_sim;

typedef struct {
  double mass[2];        /* sum over sites of rho_1, rho_2 */
  double momentum[3];    /* sum over sites of rho u = j + F/2 */
  double flow_rate;      /* (1/nx) sum rho u_x: mean mass flux through a cross-section */
  double flow_rate_disp; /* (1/nx) sum rho_1 u_x: the dispersed phase's share */
  long long step;        /* steps taken since lb_init_fields / lb_set_populations */
  long long n_interface; /* sites with |grad psi| > g_th */
  long long n_nci;       /* sites where the NCI force acts (a facing interface was hit) */
  long long n_bad;       /* sites with a non-finite or non-positive density */
} lb_obs;

/* Device bytes lb_create needs when it is given a workspace (cfg->workspace): two
 * population states of the two sets f^k_i of Eq. (CGLBE) plus scratch. */
lb_status lb_workspace_size(const lb_config* cfg, size_t* bytes);

/* Validate cfg, take the current CUDA device, allocate (or carve from the
 * workspace) two population buffers and scratch. The populations start at zero:
 * call lb_init_fields or lb_set_populations before lb_step. The model is the
 * two-component lattice Boltzmann equation, Eq. (CGLBE) of "Materials and Methods",
 * on the D2Q9 or D3Q27 lattice with the parameters of lb_config (tau of Omega^(1), A_s
 * of Omega^(2), beta of Omega^(3), A_h, h_min, h_max of Eq. (near_c)). Errors:
 * LB_EINVAL (bad configuration), LB_ENOMEM, LB_ECUDA (no usable GPU). */
lb_status lb_create(const lb_config* cfg, lb_sim** out);

/* f^k_i = f_eq_i(rho_k, u) (second-order equilibrium, c_s^2 = 1/3) at every site:
 * the state of a mixture at rest or moving with u, taken as post-collision at t = 0
 * (the densities rho_k of Eq. (CGLBE); psi = (rho1 - rho2)/(rho1 + rho2) follows).
 * rho1, rho2: [N]; u: [3][N] or NULL for u = 0. Resets the step counter. Walls come
 * from cfg->wall_y / wall_z (the channels and ducts of the paper's studies); there is
 * no per-site solid mask. Non-finite or negative values are not rejected here: they are
 * reported by the next lb_observables / lb_fields as LB_ENUMERIC. Errors: LB_EINVAL
 * (NULL rho1 or rho2), LB_ECUDA. */
lb_status lb_init_fields(lb_sim* sim, const double* rho1, const double* rho2,
                         const double* u, int on_device);

/* Advance nsteps >= 0 full steps of Eq. (CGLBE) ("Materials and Methods"): stream,
 * moments, gradient of psi, normal n and delta_I, the NCI ray and F_rep of Eq. (near_c),
 * then the collision Omega^(3)[Omega^(1) + Omega^(2)] (BGK with the force, the
 * surface-tension perturbation, recolouring). Asynchronous on cfg->stream. On the persistent TMA path
 * (lb_step_path() == LB_PATH_TMA2D) a step's launch may begin while the kernel before
 * it on the stream finishes (programmatic dependent launch); it reads and writes
 * global memory only after that kernel has completed, so results and stream order are
 * those of serial launches. Errors: LB_EINVAL (NULL sim, nsteps < 0, an ensemble
 * member), LB_ECUDA (a launch failed; the step counter stops at the last step
 * launched). */
lb_status lb_step(lb_sim* sim, long long nsteps);

/* Reductions of the current state (see lb_obs) and, optionally, psi [N] and
 * u [3][N]. flow_rate_disp, (1/nx) sum rho_1 u_x, is the periodic-channel stand-in for the
 * dispersed-phase flow rate Q_d = nu V_d of the paper's "Results" (droplets of volume
 * V_d passing at frequency nu). The macroscopic fields are those the next collision would see:
 * densities of the streamed populations and u = (j + F/2)/rho with F = G + F_rep.
 * Synchronises cfg->stream. Returns LB_ENUMERIC (with out filled) if n_bad > 0. */
lb_status lb_observables(lb_sim* sim, lb_obs* out, double* psi_out, double* u_out,
                         int on_device);

/* Per-site fields of the current state, each optional (NULL = skip):
 * rho1, rho2, psi [N]; grad psi, F_rep, u [3][N]; hit [N] = NCI distance h
 * (0 where no facing interface was found). psi and its gradient as defined after
 * Eq. (stjump), h(x) as sketched in Fig. 5, F_rep = -A_h(h) n delta_I by Eq. (near_c).
 * Synchronises cfg->stream. Returns LB_ENUMERIC (outputs filled) if a density is
 * non-finite or non-positive. */
lb_status lb_fields(lb_sim* sim, double* rho1, double* rho2, double* psi, double* grad,
                    double* frep, int* hit, double* u, int on_device);

/* Copy the populations f^k_i of Eq. (CGLBE) out of / into the sim as FP64 [2][Q][N]
 * (decoded from / encoded to the storage precision; LB_FP16DEV takes each site's reference densities as the
 * sums of the given populations). lb_set_populations resets the step counter. */
lb_status lb_get_populations(lb_sim* sim, double* f, int on_device);
lb_status lb_set_populations(lb_sim* sim, const double* f, int on_device);

/* Release everything the sim allocated. NULL is allowed. */
void lb_destroy(lb_sim* sim);

/* One-line description of the last failure on this sim (or, for sim == NULL, of
 * the last failure of lb_create / lb_workspace_size on this thread). */
const char* lb_last_error(const lb_sim* sim);

/* Step kernels launched by this sim since lb_create (for launch accounting). */
long long lb_kernel_launches(const lb_sim* sim);

/* Which kernel lb_step runs for this sim (no paper counterpart; reporting only):
 *   LB_PATH_FUSED2D  one-pass fused D2Q9 kernel (FP64; FP32 and FP16-dev when nx % 4 != 0
 *                    or LBNCI_FUSED=classic is set in the environment),
 *   LB_PATH_TMA2D    persistent TMA-fed D2Q9 kernel (FP32 and FP16-dev storage),
 *   LB_PATH_D3Q27    D3Q27 two-pass step: moments, then the collision kernel marching along
 *                    z (FP64; FP32 and FP16-dev when nx % 32 != 0 or ny % 8 != 0, or when
 *                    LBNCI_D3_KERNEL=march or tiled is set in the environment),
 *   LB_PATH_D3Q27_CARRY  D3Q27 single-read step (FP32 and FP16-dev, LBNCI_D3_KERNEL=carry): an
 *                    interface pass over densities the previous collision carried forward,
 *                    a ray pass, then a TMA-fed collision that reads each population once,
 *   LB_PATH_D3Q27_STREAM  D3Q27 streaming step (FP32 and FP16-dev on lattices of whole
 *                    32 x 8 columns: the default there): moments, per-site normals, then a
 *                    collision kernel that runs the NCI ray and needs no shared memory.
 * Returns -1 for a NULL sim. */
enum { LB_PATH_FUSED2D = 0, LB_PATH_TMA2D = 1, LB_PATH_D3Q27 = 2, LB_PATH_D3Q27_CARRY = 3, LB_PATH_D3Q27_STREAM = 4 };
int lb_step_path(const lb_sim* sim);

/* The form in which lb_step stores the state between steps (reporting only; every other
 * call sees the populations of both components whatever the form):
 *   LB_STATE_PAIRS          the populations f_i^1, f_i^2 of both components, in the
 *                           storage the precision names,
 *   LB_STATE_TOTAL_RECOLOUR streaming D3Q27 steps with Guo forcing (FP32 and FP16-dev,
 *                           unless LBNCI_D3_STATE=pairs is set in the environment when the
 *                           sim is created): the total post-collision populations
 *                           f*_i = f_i^1 + f_i^2 of the 26 moving directions, the rest
 *                           population of each component and, per site, phi_1 = rho_1/rho
 *                           and s = beta (rho_1 rho_2/rho) m, from which the recolouring
 *                           ("Materials and Methods", Omega^(3)) gives
 *                           f_i^1 = phi_1 f*_i + (w_i/|c_i|) c_i.s and f_i^2 = f*_i - f_i^1.
 *                           FP32 keeps f*_i in FP32 (128 instead of 216 bytes per site);
 *                           FP16-dev keeps f*_i - w_i rho_0 in FP16, rho_0 the mean total
 *                           density of the state as lb_init_fields or lb_set_populations set
 *                           it (76 instead of 116 bytes per site; lb_init_fields then sums
 *                           the given fields, lb_set_populations runs one fields pass, and
 *                           both synchronise the sim's stream).
 *                           The first step after a state is set reads it as pairs.
 * Returns -1 for a NULL sim. */
enum { LB_STATE_PAIRS = 0, LB_STATE_TOTAL_RECOLOUR = 1 };
int lb_state_form(const lb_sim* sim);

/* ------------------------------------------------------------------------------
 * Ensembles: n independent D2Q9 lattices of different sizes and parameters (each a
 * full lb_config: size, walls, tau, A_s, beta, A_h, h_min, h_max, g_th, force) stepped
 * together, one batched kernel launch per step for all members, replayed from a CUDA
 * graph. All members share the precision and the forcing scheme. This serves the paper's parameter studies (flow rate against the driving
 * force and the near-contact strength, "Results": Figs. 2-3) as one job. All members
 * must share the precision. The work runs on cfgs[0].stream, or on a stream of the
 * ensemble's own when that is NULL (graph capture needs a non-default stream).
 * lb_ensemble_create allocates one device block for all members (cfgs[m].workspace is
 * ignored). Each member is an ordinary lb_sim owned by the ensemble (see
 * lb_ensemble_member): every lb_* call works on it except lb_step and lb_destroy. */
typedef struct lb_ensemble lb_ensemble;

lb_status lb_ensemble_create(const lb_config* cfgs, int n, lb_ensemble** out);

/* Member m's sim handle (owned by the ensemble; valid until lb_ensemble_destroy). Use it
 * for lb_init_fields, lb_observables, lb_fields, lb_get/set_populations. */
lb_status lb_ensemble_member(lb_ensemble* ens, int m, lb_sim** out);

/* Advance every member by nsteps. Asynchronous on the ensemble's stream. */
lb_status lb_ensemble_step(lb_ensemble* ens, long long nsteps);

/* Autotuner: time the candidates of both batched kernels on the current state --
 * writing only the members' back buffers, so the state is unchanged -- and keep the
 * fastest of each. The one-pass kernel (FP64 members, nx % 4 != 0): tile shape 32 x 16
 * or 32 x 32 sites per block, *spt_out (optional) = 2 or 4. The TMA kernel (FP32 and
 * FP16-dev members with nx % 4 == 0): the L2 promotion of its tensor copies (none, 64,
 * 128, 256 bytes) x the tiles each CTA takes before it draws from the shared tile
 * counter (1, 2, 3): twelve candidates, one warm-up and five timed launches each.
 * Synchronises the ensemble's stream. */
lb_status lb_ensemble_tune(lb_ensemble* ens, int* spt_out);
/* Per-step times (ms) the last lb_ensemble_tune measured for the two shapes. */
lb_status lb_ensemble_tune_times(const lb_ensemble* ens, float* ms_32x16, float* ms_32x32);
/* The TMA kernel's current choice: *l2_promotion_bytes (0, 64, 128 or 256; 128 before
 * any tuning), *static_tiles (1, 2 or 3; 2 before any tuning), and, when ms12 is not
 * NULL, the per-step times (ms) of the last lb_ensemble_tune, ms12[ip * 3 + is] for
 * promotion index ip over {0, 64, 128, 256} and static tiles 1 + is (zero before any
 * tuning). Any pointer may be NULL. LB_EUNSUPPORTED when no member runs that kernel. */
lb_status lb_ensemble_tma_choice(const lb_ensemble* ens, int* l2_promotion_bytes, int* static_tiles, float* ms12);

/* Batched step launches since creation; last failure on this ensemble. */
long long lb_ensemble_launches(const lb_ensemble* ens);
const char* lb_ensemble_last_error(const lb_ensemble* ens);

/* Release the ensemble and all its members. NULL is allowed. */
void lb_ensemble_destroy(lb_ensemble* ens);

/* Observables with no allocation at all. The paper has no counterpart: this is a
 * convenience for callers that cannot let a library allocate device memory (an
 * application whose device memory is fully reserved by its own pool allocator; a loop
 * that must not risk the device synchronisation a cudaMalloc can cause).
 * Computes exactly what lb_observables reports (step is set to 0) for the caller's
 * populations f: a device array [2][Q][N] in the storage type of cfg->precision
 * (double for LB_FP64, float for LB_FP32), laid out as lb_get_populations describes.
 * cfg->workspace is ignored; work runs on cfg->stream, and the call copies its result
 * to the host and synchronises cfg->stream before it returns, so it cannot be made while
 * cfg->stream is being captured into a CUDA graph (between captured segments it adds no
 * allocation).
 * Scratch comes from a fixed 8 MiB static device array inside the library (held by
 * every GPU that loads it until the process exits), so lattices are limited to about
 * 2 million sites in FP32 and 1 million in FP64; larger ones return LB_EINVAL with
 * the sizes in lb_last_error(NULL). Every call looks up the array's device address on
 * the current device (the first call on a device may load the library's device code).
 * All calls share the array: calls that overlap on the GPU (other streams, other host
 * threads on the same device) race and must not be issued. Returns LB_ENUMERIC (with
 * out filled) if n_bad > 0. */
lb_status lb_observables_noalloc(const lb_config* cfg, const void* f, lb_obs* out);

#ifdef __cplusplus
}
#endif
#endif
