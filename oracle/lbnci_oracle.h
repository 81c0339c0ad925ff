/*
 * lbnci_oracle.h -- FP64 CPU oracle of the two-component colour-gradient lattice
 * Boltzmann step with the near-contact-interaction (NCI) force of
 * Montessori et al., "Lattice Boltzmann simulations capture the multiscale physics
 * of soft flowing crystals" (arXiv:2003.11069), section "Materials and Methods".
 *
 * TEST INFRASTRUCTURE. This library is the slow, obviously-correct judge of the
 * CUDA path. Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it. It shares no code, header, table or constant with the CUDA
 * library: every table below is generated here from its definition.
 *
 * Conventions (stated independently in the public CUDA header as well):
 *   - site index  idx = x + nx*(y + ny*z)    (x fastest; nz = 1 on D2Q9)
 *   - populations f[k][i][idx], k = 0 (component 1, dispersed, psi > 0) or 1,
 *     i = 0..Q-1 with c_i given by the base-3 digits of i, digit d -> {0,+1,-1}[d]
 *     (x from the lowest digit, then y, then z).
 *   - the stored state between steps is the post-collision population at its
 *     own site; a step pulls (streams) first and then collides.
 */
#ifndef LBNCI_ORACLE_H
#define LBNCI_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int lattice;   /* 0 = D2Q9, 1 = D3Q27 */
  int nx, ny, nz;
  int wall_y;    /* 1: halfway bounce-back walls below y=0 and above y=ny-1; 0: periodic */
  int wall_z;    /* same along z (D3Q27 only) */
  double tau;    /* BGK relaxation time of the mixture */
  double A_s;    /* perturbation (surface-tension) amplitude of each component */
  double beta;   /* recolouring segregation parameter */
  double A_h;    /* NCI strength constant A */
  double h_min, h_max; /* NCI cut-offs in lattice units */
  double g_th;   /* |grad psi| above which a site belongs to an interface */
  double force[3]; /* uniform body-force density G */
  int forcing;   /* 0: Guo forcing of the mixture; 1: exact difference method with the
                    NCI force on the dispersed phase only (see lbnci_oracle.c) */
} orc_params;

/* Lattice tables: c[Q][3], w[Q], opp[Q]. Returns Q, or -1 for an unknown lattice. */
int orc_lattice(int lattice, int* c, double* w, int* opp);

/* f <- f_eq(rho_k, u) for both components; u is [3][N] or NULL (u = 0). */
int orc_init(const orc_params* p, const double* rho1, const double* rho2,
             const double* u, double* f);

/* Advance f (the post-collision state, [2][Q][N]) by nsteps full steps. */
int orc_step(const orc_params* p, double* f, long nsteps, int nthreads);

/* Macroscopic fields the next collision sees: pulled densities, order parameter,
 * isotropic gradient [3][N], NCI force [3][N], NCI hit distance h (0 = none) and
 * the Guo velocity u = (j + F/2)/rho [3][N]. Any output pointer may be NULL. */
int orc_fields(const orc_params* p, const double* f, double* rho1, double* rho2,
               double* psi, double* grad, double* frep, int* hit, double* u);

/* out[7] = {mass_1, mass_2, P_x, P_y, P_z, Q_tot, Q_disp} (see orc_fields). */
int orc_observables(const orc_params* p, const double* f, double* out);

/* Isotropic gradient of a given psi field (walls mirror the centre value). */
int orc_gradient(const orc_params* p, const double* psi, double* grad);

/* NCI force and hit distance of a given psi field. */
int orc_nci(const orc_params* p, const double* psi, double* frep, int* hit);

/* One site's collision + recolouring: fin[2][Q] pulled populations, the
 * gradient of psi at the site and the total force F; writes fout[2][Q]. */
int orc_collide_site(const orc_params* p, const double* fin, const double* grad,
                     const double* F, double* fout);

#ifdef __cplusplus
}
#endif
#endif
