/*
 * lbnci_oracle.c -- plain FP64 CPU oracle of one time step of the two-component
 * colour-gradient lattice Boltzmann method with near-contact interactions (NCI)
 * of Montessori et al., arXiv:2003.11069, "Materials and Methods".
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path. Nested loops, no
 * blocking, no fusion, stages in the paper's order. Compile with
 * -O2 -ffp-contract=off so that no multiply-add is contracted.
 *
 * A step, from the post-collision state f* of the previous step:
 *   1. stream (pull) with halfway bounce-back at walls            Eq. (CGLBE)
 *   2. moments rho_k = sum_i f_i^k, psi = (rho1-rho2)/(rho1+rho2)  (moments; psi def.)
 *   3. isotropic 2nd-order gradient of psi, |grad psi|, normal n = -grad psi/|grad psi|,
 *      delta_I = |grad psi|/2                                      (n and delta_I defs.)
 *   4. NCI: distance h to a facing interface along n, A_h(h), F_rep = -A_h(h) n delta_I
 *                                                                   Eq. (near_c)
 *   5. force F = G + F_rep, Guo velocity u = (j + F/2)/rho
 *   6. Omega^(1) BGK + Guo source, Omega^(2) perturbation on the total f
 *   7. Omega^(3) recolouring into the two components               (collision operator)
 *
 * Readings where the paper is silent (each also stated in the design notes):
 *   - relaxation form: single-time BGK with Guo forcing (the paper inserts the
 *     force with the exact difference method; the hot path uses Guo);
 *   - perturbation: (A_s/2)|grad psi| [w_i (c_i.m)^2 - B_i] per component,
 *     m = grad psi/|grad psi|, B_i = w_i/3, same A_s for both components;
 *   - recolouring: f^1 = (rho1/rho) f + beta (rho1 rho2/rho) w_i cos(theta_i),
 *     f^2 = (rho2/rho) f - same, cos(theta_i) = c_i.m/|c_i| (0 for the rest vector);
 *   - walls: a solid neighbour contributes the psi of its mirror image across the
 *     wall plane to the gradient (neutral wetting);
 *   - forcing = 1 (the paper's own insertion of the force, end of "Materials and
 *     Methods": exact difference method, NCI force on the dispersed phase only): the
 *     relaxation uses u = j/rho; after recolouring component k gains
 *     f_eq_i(rho_k, u + dU_k) - f_eq_i(rho_k, u), dU_k = F_k/rho_k, with
 *     F_1 = G rho_1/rho + F_rep and F_2 = G rho_2/rho (the body force acts on the
 *     mixture in proportion to mass); the reported velocity is still (j + F/2)/rho;
 *   - NCI ray: x is an interface site when |grad psi| > g_th; for s = 1..floor(h_max)
 *     the probe y = x + round(s n) (round half away from zero per component);
 *     a probe in a wall ends the search; the first probe with |grad psi(y)| > g_th
 *     and n(y).n(x) < 0 is the hit, h = s; A_h(h) = A for h <= h_min,
 *     A (h_min/h)^3 for h_min < h <= h_max, 0 beyond.
 */
#include "lbnci_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QMAX 27

typedef struct {
  int D, Q;
  int c[QMAX][3];
  double w[QMAX];
  int opp[QMAX];
  double inv_len[QMAX];
} lattice_t;

/* Base-3 digit d of the direction index maps to the velocity component {0,+1,-1}[d]. */
static int digit_to_c(int d) { return d == 0 ? 0 : (d == 1 ? 1 : -1); }

static int make_lattice(int lattice, lattice_t* L) {
  if (lattice == 0) { L->D = 2; L->Q = 9; }
  else if (lattice == 1) { L->D = 3; L->Q = 27; }
  else return -1;
  for (int i = 0; i < L->Q; ++i) {
    L->c[i][0] = digit_to_c(i % 3);
    L->c[i][1] = digit_to_c((i / 3) % 3);
    L->c[i][2] = digit_to_c(i / 9);
    int c2 = L->c[i][0] * L->c[i][0] + L->c[i][1] * L->c[i][1] + L->c[i][2] * L->c[i][2];
    /* Standard weights of the D2Q9 and D3Q27 lattices, by speed |c|^2. */
    if (L->D == 2) {
      const double w2[3] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 36.0};
      L->w[i] = w2[c2];
    } else {
      const double w3[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
      L->w[i] = w3[c2];
    }
    L->inv_len[i] = c2 == 0 ? 0.0 : 1.0 / sqrt((double)c2);
  }
  for (int i = 0; i < L->Q; ++i)
    for (int j = 0; j < L->Q; ++j)
      if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
        L->opp[i] = j;
  return 0;
}

int orc_lattice(int lattice, int* c, double* w, int* opp) {
  lattice_t L;
  if (make_lattice(lattice, &L)) return -1;
  for (int i = 0; i < L.Q; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = L.c[i][a];
    w[i] = L.w[i];
    opp[i] = L.opp[i];
  }
  return L.Q;
}

static long nsites(const orc_params* p) { return (long)p->nx * p->ny * p->nz; }

static int check_params(const orc_params* p, lattice_t* L) {
  if (make_lattice(p->lattice, L)) return -1;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
  if (L->D == 2 && p->nz != 1) return -1;
  return 0;
}

/* Index of the site (x,y,z)+d, or -1 when it lies beyond a wall. x is always
 * periodic; y and z are periodic unless walled. */
static long neighbour(const orc_params* p, int x, int y, int z, int dx, int dy, int dz) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  X = ((X % p->nx) + p->nx) % p->nx;
  if (p->wall_y) { if (Y < 0 || Y >= p->ny) return -1; }
  else Y = ((Y % p->ny) + p->ny) % p->ny;
  if (p->nz > 1 && p->wall_z) { if (Z < 0 || Z >= p->nz) return -1; }
  else Z = ((Z % p->nz) + p->nz) % p->nz;
  return (long)X + (long)p->nx * ((long)Y + (long)p->ny * Z);
}

static void site_xyz(const orc_params* p, long idx, int* x, int* y, int* z) {
  *x = (int)(idx % p->nx);
  *y = (int)((idx / p->nx) % p->ny);
  *z = (int)(idx / ((long)p->nx * p->ny));
}

/* Equilibrium of the second-order lattice BGK model, c_s^2 = 1/3. */
static double feq(const lattice_t* L, int i, double rho, const double u[3]) {
  double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

int orc_init(const orc_params* p, const double* rho1, const double* rho2,
             const double* u, double* f) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
  long N = nsites(p);
  for (long s = 0; s < N; ++s) {
    double us[3] = {0.0, 0.0, 0.0};
    if (u) { us[0] = u[s]; us[1] = u[N + s]; us[2] = u[2 * N + s]; }
    for (int i = 0; i < L.Q; ++i) {
      f[(0 * L.Q + i) * N + s] = feq(&L, i, rho1[s], us);
      f[(1 * L.Q + i) * N + s] = feq(&L, i, rho2[s], us);
    }
  }
  return 0;
}

/* Stage 1: pull streaming with halfway bounce-back. */
static void stream(const orc_params* p, const lattice_t* L, const double* f, double* fp) {
  long N = nsites(p);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < N; ++s) {
    int x, y, z;
    site_xyz(p, s, &x, &y, &z);
    for (int i = 0; i < L->Q; ++i) {
      long src = neighbour(p, x, y, z, -L->c[i][0], -L->c[i][1], -L->c[i][2]);
      for (int k = 0; k < 2; ++k) {
        if (src >= 0) fp[(k * L->Q + i) * N + s] = f[(k * L->Q + i) * N + src];
        else fp[(k * L->Q + i) * N + s] = f[(k * L->Q + L->opp[i]) * N + s];
      }
    }
  }
}

/* Stage 2: component densities and order parameter. */
static void moments(const orc_params* p, const lattice_t* L, const double* fp,
                    double* rho1, double* rho2, double* psi) {
  long N = nsites(p);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < N; ++s) {
    double r[2] = {0.0, 0.0};
    for (int k = 0; k < 2; ++k)
      for (int i = 0; i < L->Q; ++i) r[k] += fp[(k * L->Q + i) * N + s];
    rho1[s] = r[0];
    rho2[s] = r[1];
    psi[s] = (r[0] - r[1]) / (r[0] + r[1]);
  }
}

/* Stage 3: grad psi(x) = (1/c_s^2) sum_i w_i c_i psi(x + c_i). A neighbour beyond a
 * wall takes the value of its mirror image across the wall plane: the site reached
 * by dropping the velocity components that cross the wall (neutral wetting). */
static long mirrored_neighbour(const orc_params* p, int x, int y, int z, const int c[3]) {
  int d[3] = {c[0], c[1], c[2]};
  if (p->wall_y && (y + d[1] < 0 || y + d[1] >= p->ny)) d[1] = 0;
  if (p->nz > 1 && p->wall_z && (z + d[2] < 0 || z + d[2] >= p->nz)) d[2] = 0;
  return neighbour(p, x, y, z, d[0], d[1], d[2]);
}

static void gradient(const orc_params* p, const lattice_t* L, const double* psi, double* grad) {
  long N = nsites(p);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < N; ++s) {
    int x, y, z;
    site_xyz(p, s, &x, &y, &z);
    double g[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->Q; ++i) {
      double v = psi[mirrored_neighbour(p, x, y, z, L->c[i])];
      for (int a = 0; a < 3; ++a) g[a] += L->w[i] * L->c[i][a] * v;
    }
    for (int a = 0; a < 3; ++a) grad[a * N + s] = 3.0 * g[a];
  }
}

/* Round half away from zero (exact; C99 round). */
static int round_away(double v) { return (int)round(v); }

/* NCI strength profile A_h(h). */
static double nci_strength(const orc_params* p, int h) {
  double hd = (double)h;
  if (hd <= p->h_min) return p->A_h;
  if (hd <= p->h_max) {
    double r = p->h_min / hd;
    return p->A_h * (r * r * r);
  }
  return 0.0;
}

static double norm3(const double* grad, long N, long s) {
  double gx = grad[s], gy = grad[N + s], gz = grad[2 * N + s];
  return sqrt(gx * gx + gy * gy + gz * gz);
}

/* Stage 4: NCI force F_rep = -A_h(h) n delta_I at interface sites, with
 * n = -grad psi/|grad psi| and delta_I = |grad psi|/2. */
static void nci(const orc_params* p, const lattice_t* L, const double* grad,
                double* frep, int* hit) {
  long N = nsites(p);
  int smax = (int)floor(p->h_max);
#pragma omp parallel for schedule(static)
  for (long s = 0; s < N; ++s) {
    for (int a = 0; a < 3; ++a) frep[a * N + s] = 0.0;
    if (hit) hit[s] = 0;
    double g = norm3(grad, N, s);
    if (!(g > p->g_th)) continue;
    double n[3];
    for (int a = 0; a < 3; ++a) n[a] = -grad[a * N + s] / g;
    int x, y, z;
    site_xyz(p, s, &x, &y, &z);
    int h = 0;
    for (int step = 1; step <= smax; ++step) {
      int d[3];
      for (int a = 0; a < 3; ++a) d[a] = round_away(step * n[a]);
      if (L->D == 2) d[2] = 0;
      long ys = neighbour(p, x, y, z, d[0], d[1], d[2]);
      if (ys < 0) break;
      double gy = norm3(grad, N, ys);
      if (!(gy > p->g_th)) continue;
      double dot = 0.0;
      for (int a = 0; a < 3; ++a) dot += (-grad[a * N + ys] / gy) * n[a];
      if (dot < 0.0) { h = step; break; }
    }
    if (h == 0) continue;
    if (hit) hit[s] = h;
    double A = nci_strength(p, h);
    double deltaI = 0.5 * g;
    for (int a = 0; a < 3; ++a) frep[a * N + s] = -A * n[a] * deltaI;
  }
}

/* Stages 5-7 at one site: BGK + Guo source + perturbation on the total
 * population, then recolouring. fin is [2][Q] with stride `st`, fout with `so`.
 * With forcing = 1 the force enters instead by the exact difference method after
 * recolouring (see the header comment). */
static void collide(const orc_params* p, const lattice_t* L, const double* fin, long st,
                    const double grad[3], const double F[3], double* fout, long so,
                    double* u_out) {
  int Q = L->Q;
  double rho1 = 0.0, rho2 = 0.0;
  for (int i = 0; i < Q; ++i) rho1 += fin[i * st];
  for (int i = 0; i < Q; ++i) rho2 += fin[(Q + i) * st];
  double rho = rho1 + rho2;
  double j[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; ++i) {
    double fi = fin[i * st] + fin[(Q + i) * st];
    for (int a = 0; a < 3; ++a) j[a] += fi * L->c[i][a];
  }
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
  if (u_out) for (int a = 0; a < 3; ++a) u_out[a] = u[a];
  const int edm = p->forcing == 1;
  double ueq[3];  /* velocity of the equilibrium the populations relax to */
  for (int a = 0; a < 3; ++a) ueq[a] = edm ? j[a] / rho : u[a];

  double g = sqrt(grad[0] * grad[0] + grad[1] * grad[1] + grad[2] * grad[2]);
  double m[3] = {0.0, 0.0, 0.0}; /* unit colour gradient, grad psi/|grad psi| */
  if (g > 0.0) for (int a = 0; a < 3; ++a) m[a] = grad[a] / g;

  double omega = 1.0 / p->tau;
  double guo = 1.0 - 0.5 * omega;
  double uF = u[0] * F[0] + u[1] * F[1] + u[2] * F[2];
  double seg = p->beta * rho1 * rho2 / rho;
  /* exact difference method: velocity shift of each component */
  double dU[2][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
  if (edm) {
    for (int a = 0; a < 3; ++a) {
      double G = p->force[a], Frep = F[a] - p->force[a];
      if (rho1 > 0.0) dU[0][a] = (G * rho1 / rho + Frep) / rho1;
      if (rho2 > 0.0) dU[1][a] = (G * rho2 / rho) / rho2;
    }
  }
  for (int i = 0; i < Q; ++i) {
    double fi = fin[i * st] + fin[(Q + i) * st];
    double cu = L->c[i][0] * u[0] + L->c[i][1] * u[1] + L->c[i][2] * u[2];
    double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
    double cm = L->c[i][0] * m[0] + L->c[i][1] * m[1] + L->c[i][2] * m[2];
    double fs;
    if (!edm) {
      /* Omega^(1): BGK towards f_eq(rho, u), plus the Guo source term. */
      double S = guo * L->w[i] * (3.0 * (cF - uF) + 9.0 * cu * cF);
      fs = fi - omega * (fi - feq(L, i, rho, u)) + S;
    } else {
      fs = fi - omega * (fi - feq(L, i, rho, ueq));
    }
    /* Omega^(2): perturbation, summed over the two components. */
    double pert = 2.0 * (0.5 * p->A_s) * g * (L->w[i] * cm * cm - L->w[i] / 3.0);
    fs += pert;
    /* Omega^(3): recolouring. */
    double cos_t = cm * L->inv_len[i];
    double rc = seg * L->w[i] * cos_t;
    double o1 = rho1 / rho * fs + rc;
    double o2 = rho2 / rho * fs - rc;
    if (edm) {
      /* forcing: f_eq(rho_k, u + dU_k) - f_eq(rho_k, u) for each component */
      double u1[3], u2[3];
      for (int a = 0; a < 3; ++a) { u1[a] = ueq[a] + dU[0][a]; u2[a] = ueq[a] + dU[1][a]; }
      o1 += feq(L, i, rho1, u1) - feq(L, i, rho1, ueq);
      o2 += feq(L, i, rho2, u2) - feq(L, i, rho2, ueq);
    }
    fout[i * so] = o1;
    fout[(Q + i) * so] = o2;
  }
}

int orc_collide_site(const orc_params* p, const double* fin, const double* grad,
                     const double* F, double* fout) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
  collide(p, &L, fin, 1, grad, F, fout, 1, NULL);
  return 0;
}

typedef struct {
  double *fp, *rho1, *rho2, *psi, *grad, *frep;
  int* hit;
} work_t;

static int work_alloc(long N, int Q, work_t* w) {
  w->fp = malloc(sizeof(double) * 2 * Q * N);
  w->rho1 = malloc(sizeof(double) * N);
  w->rho2 = malloc(sizeof(double) * N);
  w->psi = malloc(sizeof(double) * N);
  w->grad = malloc(sizeof(double) * 3 * N);
  w->frep = malloc(sizeof(double) * 3 * N);
  w->hit = malloc(sizeof(int) * N);
  return (w->fp && w->rho1 && w->rho2 && w->psi && w->grad && w->frep && w->hit) ? 0 : -1;
}

static void work_free(work_t* w) {
  free(w->fp); free(w->rho1); free(w->rho2); free(w->psi);
  free(w->grad); free(w->frep); free(w->hit);
}

/* Stages 1-4 of a step, leaving pulled populations and fields in w. */
static void prepare(const orc_params* p, const lattice_t* L, const double* f, work_t* w) {
  stream(p, L, f, w->fp);
  moments(p, L, w->fp, w->rho1, w->rho2, w->psi);
  gradient(p, L, w->psi, w->grad);
  nci(p, L, w->grad, w->frep, w->hit);
}

static void total_force(const orc_params* p, const double* frep, long N, long s, double F[3]) {
  for (int a = 0; a < 3; ++a) F[a] = p->force[a] + frep[a * N + s];
}

#ifdef _OPENMP
#include <omp.h>
#endif

int orc_step(const orc_params* p, double* f, long nsteps, int nthreads) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  long N = nsites(p);
  work_t w;
  if (work_alloc(N, L.Q, &w)) { work_free(&w); return -2; }
  for (long t = 0; t < nsteps; ++t) {
    prepare(p, &L, f, &w);
#pragma omp parallel for schedule(static)
    for (long s = 0; s < N; ++s) {
      double grad[3] = {w.grad[s], w.grad[N + s], w.grad[2 * N + s]};
      double F[3];
      total_force(p, w.frep, N, s, F);
      collide(p, &L, w.fp + s, N, grad, F, f + s, N, NULL);
    }
  }
  work_free(&w);
  return 0;
}

int orc_fields(const orc_params* p, const double* f, double* rho1, double* rho2,
               double* psi, double* grad, double* frep, int* hit, double* u) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
  long N = nsites(p);
  work_t w;
  if (work_alloc(N, L.Q, &w)) { work_free(&w); return -2; }
  prepare(p, &L, f, &w);
  if (rho1) memcpy(rho1, w.rho1, sizeof(double) * N);
  if (rho2) memcpy(rho2, w.rho2, sizeof(double) * N);
  if (psi) memcpy(psi, w.psi, sizeof(double) * N);
  if (grad) memcpy(grad, w.grad, sizeof(double) * 3 * N);
  if (frep) memcpy(frep, w.frep, sizeof(double) * 3 * N);
  if (hit) memcpy(hit, w.hit, sizeof(int) * N);
  if (u) {
    double* tmp = malloc(sizeof(double) * 2 * L.Q);
    for (long s = 0; s < N; ++s) {
      double g3[3] = {w.grad[s], w.grad[N + s], w.grad[2 * N + s]};
      double F[3], us[3];
      total_force(p, w.frep, N, s, F);
      collide(p, &L, w.fp + s, N, g3, F, tmp, 1, us);
      for (int a = 0; a < 3; ++a) u[a * N + s] = us[a];
    }
    free(tmp);
  }
  work_free(&w);
  return 0;
}

/* Compensated (Kahan) accumulation in site order. */
typedef struct { double s, c; } ksum;
static void kadd(ksum* k, double v) {
  double y = v - k->c;
  double t = k->s + y;
  k->c = (t - k->s) - y;
  k->s = t;
}

int orc_observables(const orc_params* p, const double* f, double* out) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
  long N = nsites(p);
  double* rho1 = malloc(sizeof(double) * N);
  double* rho2 = malloc(sizeof(double) * N);
  double* u = malloc(sizeof(double) * 3 * N);
  if (!rho1 || !rho2 || !u) { free(rho1); free(rho2); free(u); return -2; }
  int rc = orc_fields(p, f, rho1, rho2, NULL, NULL, NULL, NULL, u);
  if (rc) { free(rho1); free(rho2); free(u); return rc; }
  ksum acc[7];
  memset(acc, 0, sizeof(acc));
  for (long s = 0; s < N; ++s) {
    double rho = rho1[s] + rho2[s];
    kadd(&acc[0], rho1[s]);
    kadd(&acc[1], rho2[s]);
    for (int a = 0; a < 3; ++a) kadd(&acc[2 + a], rho * u[a * N + s]);
    kadd(&acc[5], rho * u[s]);
    kadd(&acc[6], rho1[s] * u[s]);
  }
  for (int q = 0; q < 7; ++q) out[q] = acc[q].s;
  out[5] /= (double)p->nx; /* mean mass flux through one cross-section */
  out[6] /= (double)p->nx;
  free(rho1); free(rho2); free(u);
  return 0;
}

int orc_gradient(const orc_params* p, const double* psi, double* grad) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
  gradient(p, &L, psi, grad);
  return 0;
}

int orc_nci(const orc_params* p, const double* psi, double* frep, int* hit) {
  lattice_t L;
  if (check_params(p, &L)) return -1;
  long N = nsites(p);
  double* grad = malloc(sizeof(double) * 3 * N);
  if (!grad) return -2;
  gradient(p, &L, psi, grad);
  nci(p, &L, grad, frep, hit);
  free(grad);
  return 0;
}
