/* pt_oracle.c — plain FP64 CPU oracle of the pseudo-transient (PT) + Picard solver for 3-D
 * nonlinear poroviscoelastic two-phase flow.
 *
 * TEST INFRASTRUCTURE ONLY: the CUDA path is checked against this file. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every step below is one plain loop over one staggered array, written straight from the
 * formulas, in the order of one PT iteration k -> k+1:
 *   1. coefficients from phi^k            k = k0 e^theta (phi/phi0)^3 (Eq. 23), rho g (Eq. 27)
 *   2. Darcy flux and its divergence      Eq. 20 with zero normal flux on the boundary (Eq. 34)
 *   3. div V and the numerical div V      left-hand side of Eq. 17
 *   4. local-implicit pressure updates    Eqs. 17-18 (pseudo-time steps of the appendix script)
 *   5. Maxwell viscoelastic stresses      Eq. 21 in backward-Euler form (not stored per iteration)
 *   6. damped momentum residual           Eq. 19 with the velocity damping of Section 2.2
 *   7. porosity in log space              Eq. 22 (log(1 - phi) form, Section 2.2)
 *   8. velocity update, free slip         normal velocity 0 on the boundary
 *   9. Picard update (every nup-th)       Eqs. 24-26 with log-space relaxation
 *  10. residual max-norms (every nup-th)  convergence test
 * Parity unpinned: the thesis prints no field values for this solver; the tests pin the oracle
 * to closed forms, invariants and a brute-force Newton solve instead.
 */
#include "pt_oracle.h"

#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- indexing (x fastest) */
#define NX (p->nx)
#define NY (p->ny)
#define NZ (p->nz)
#define C_(i, j, k)   ((long)(i) + (long)NX * ((long)(j) + (long)NY * (long)(k)))
#define FX_(i, j, k)  ((long)(i) + (long)(NX + 1) * ((long)(j) + (long)NY * (long)(k)))
#define FY_(i, j, k)  ((long)(i) + (long)NX * ((long)(j) + (long)(NY + 1) * (long)(k)))
#define FZ_(i, j, k)  ((long)(i) + (long)NX * ((long)(j) + (long)NY * (long)(k)))
#define EXY_(i, j, k) ((long)(i) + (long)(NX + 1) * ((long)(j) + (long)(NY + 1) * (long)(k)))
#define EXZ_(i, j, k) ((long)(i) + (long)(NX + 1) * ((long)(j) + (long)NY * (long)(k)))
#define EYZ_(i, j, k) ((long)(i) + (long)NX * ((long)(j) + (long)(NY + 1) * (long)(k)))

static long n_centre(const or_params *p) { return (long)NX * NY * NZ; }
static long n_fx(const or_params *p) { return (long)(NX + 1) * NY * NZ; }
static long n_fy(const or_params *p) { return (long)NX * (NY + 1) * NZ; }
static long n_fz(const or_params *p) { return (long)NX * NY * (NZ + 1); }
static long n_exy(const or_params *p) { return (long)(NX + 1) * (NY + 1) * NZ; }
static long n_exz(const or_params *p) { return (long)(NX + 1) * NY * (NZ + 1); }
static long n_eyz(const or_params *p) { return (long)NX * (NY + 1) * (NZ + 1); }

static double h_x(const or_params *p) { return p->lx / NX; }
static double h_y(const or_params *p) { return p->ly / NY; }
static double h_z(const or_params *p) { return p->lz / NZ; }
static double h_min2(const or_params *p) {
  double h = fmin(h_x(p), fmin(h_y(p), h_z(p)));
  return h * h;
}
/* background density times gravity, rho_BG g = phi0 rho_f g + (1 - phi0) rho_s g (Eq. 27 at phi0);
 * pressures are excess over the lithostatic pressure of this background. */
static double rho_bg_g(const or_params *p) { return p->phi0 * p->rhof_g + (1.0 - p->phi0) * p->rhos_g; }

static int params_ok(const or_params *p) {
  if (!p) return 0;
  if (NX < 1 || NY < 1 || NZ < 1) return 0;
  if (!(p->lx > 0 && p->ly > 0 && p->lz > 0)) return 0;
  if (!(p->dt > 0) || p->nup < 1 || p->max_iter < 0) return 0;
  if (!(p->phi0 > 0 && p->phi0 < 1) || !(p->mu0 > 0) || !(p->eta0 > 0) || !(p->k0 > 0)) return 0;
  if (!(p->G > 0) || !(p->rho_i > 0) || !(p->alpha > 0) || !(p->B > 0)) return 0;
  if (!(p->xsi_w > 0)) return 0;
  return 1;
}

/* ------------------------------------------------------------ step 1: coefficients */
void or_coefficients(const or_params *p, const double *phi, const double *logk,
                     double *perm, double *rog) {
  const double rbg = rho_bg_g(p);
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double ph = phi[c];
        const double th = logk ? logk[c] : 0.0;
        const double r = ph / p->phi0;
        perm[c] = p->k0 * exp(th) * r * r * r;                       /* Eq. 23, k / mu_f */
        rog[c] = (ph * p->rhof_g + (1.0 - ph) * p->rhos_g) - rbg;    /* Eq. 27, excess   */
      }
}

/* ------------------------------------------------------ step 2: Darcy flux, Eq. 20 */
void or_darcy(const or_params *p, const double *Pf, const double *perm,
              double *qx, double *qy, double *qz, double *divqD) {
  const double dx = h_x(p), dy = h_y(p), dz = h_z(p);
  const double buoy = p->rhof_g - rho_bg_g(p);   /* (rho_f - rho_BG) g, gravity along -z */
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i <= NX; ++i) {
        double q = 0.0;                          /* zero normal flux on the boundary (Eq. 34) */
        if (i > 0 && i < NX) {
          const double kf = 0.5 * (perm[C_(i - 1, j, k)] + perm[C_(i, j, k)]);
          q = -kf * (Pf[C_(i, j, k)] - Pf[C_(i - 1, j, k)]) / dx;
        }
        qx[FX_(i, j, k)] = q;
      }
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j <= NY; ++j)
      for (int i = 0; i < NX; ++i) {
        double q = 0.0;
        if (j > 0 && j < NY) {
          const double kf = 0.5 * (perm[C_(i, j - 1, k)] + perm[C_(i, j, k)]);
          q = -kf * (Pf[C_(i, j, k)] - Pf[C_(i, j - 1, k)]) / dy;
        }
        qy[FY_(i, j, k)] = q;
      }
#pragma omp parallel for
  for (int k = 0; k <= NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        double q = 0.0;
        if (k > 0 && k < NZ) {
          const double kf = 0.5 * (perm[C_(i, j, k - 1)] + perm[C_(i, j, k)]);
          q = -kf * ((Pf[C_(i, j, k)] - Pf[C_(i, j, k - 1)]) / dz + buoy);
        }
        qz[FZ_(i, j, k)] = q;
      }
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i)
        divqD[C_(i, j, k)] = (qx[FX_(i + 1, j, k)] - qx[FX_(i, j, k)]) / dx +
                             (qy[FY_(i, j + 1, k)] - qy[FY_(i, j, k)]) / dy +
                             (qz[FZ_(i, j, k + 1)] - qz[FZ_(i, j, k)]) / dz;
}

/* pseudo-time step of the solid velocity at a centre (averaged to faces):
 * dtau_V = cfl_v h^2 rho_i / (mu (1 + beta_n)), the appendix script's form with its velocity
 * scale 1 / (1 + beta_n) as a factor */
static double dtau_v(const or_params *p, double mu) {
  return p->cfl_v * h_min2(p) * p->rho_i / (mu * (1.0 + p->beta_n));
}

/* compaction coefficient 1 / (eta (1 - phi)) of Eqs. 17-18, zero when compaction is off */
static double compaction_coef(const or_params *p, double eta, double phi) {
  return p->compaction_on ? 1.0 / (eta * (1.0 - phi)) : 0.0;
}

/* -------------------------------------- step 3: div V and numerical div V (Eq. 17 LHS) */
void or_divergence(const or_params *p, const double *Vx, const double *Vy, const double *Vz,
                   const double *Pt, const double *Pf, const double *Pto, const double *Pfo,
                   const double *phi, const double *eta, double *divV, double *divVn) {
  const double dx = h_x(p), dy = h_y(p), dz = h_z(p);
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double dv = (Vx[FX_(i + 1, j, k)] - Vx[FX_(i, j, k)]) / dx +
                          (Vy[FY_(i, j + 1, k)] - Vy[FY_(i, j, k)]) / dy +
                          (Vz[FZ_(i, j, k + 1)] - Vz[FZ_(i, j, k)]) / dz;
        divV[c] = dv;
        divVn[c] = dv + p->beta_d * ((Pt[c] - Pto[c]) - p->alpha * (Pf[c] - Pfo[c])) / p->dt +
                   (Pt[c] - Pf[c]) * compaction_coef(p, eta[c], phi[c]);
      }
}

/* fluid-pressure residual of Eq. 18 (sign of the appendix script: descent direction) */
static double pf_residual(const or_params *p, double divqD, double Pt, double Pf, double Pto,
                          double Pfo, double eta, double phi) {
  return divqD + p->beta_d * p->alpha * ((Pf - Pfo) / p->B - (Pt - Pto)) / p->dt +
         (Pf - Pt) * compaction_coef(p, eta, phi);
}

/* -------------------------------------------- step 4: local-implicit pressure updates */
static void pressure_update(const or_params *p, const or_state *s, const double *perm,
                            const double *divV, const double *divqD, double *Pt1, double *Pf1) {
  const double h2 = h_min2(p);
  const double dt = p->dt, bd = p->beta_d, al = p->alpha, B = p->B;
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double Pt = s->Pt[c], Pf = s->Pf[c], Pto = s->Pto[c], Pfo = s->Pfo[c];
        const double cc = compaction_coef(p, s->eta[c], s->phi[c]);
        /* largest permeability of the cell and its existing face neighbours */
        double kmax = perm[c];
        if (i > 0) kmax = fmax(kmax, perm[C_(i - 1, j, k)]);
        if (i < NX - 1) kmax = fmax(kmax, perm[C_(i + 1, j, k)]);
        if (j > 0) kmax = fmax(kmax, perm[C_(i, j - 1, k)]);
        if (j < NY - 1) kmax = fmax(kmax, perm[C_(i, j + 1, k)]);
        if (k > 0) kmax = fmax(kmax, perm[C_(i, j, k - 1)]);
        if (k < NZ - 1) kmax = fmax(kmax, perm[C_(i, j, k + 1)]);
        const double dtau_pt = p->dtpt_scale * s->mu[c] * (1.0 + p->beta_n) / NZ;
        const double dtau_pf = p->cfl_pf * h2 * (1.0 + bd * B / al) / kmax;
        /* Pt^{k+1} = Pt - dtau (div V + beta_d (Pt^{k+1} - Pto - al (Pf - Pfo)) / dt
         *                      + (Pt^{k+1} - Pf) cc),  solved for Pt^{k+1}             */
        Pt1[c] = (Pt - dtau_pt * (divV[c] + bd * (-Pto - al * (Pf - Pfo)) / dt - cc * Pf)) /
                 (1.0 + dtau_pt * (bd / dt + cc));
        /* Pf^{k+1} = Pf - dtau (div qD + bd al ((Pf^{k+1} - Pfo) / B - (Pt - Pto)) / dt
         *                      + (Pf^{k+1} - Pt) cc),  solved for Pf^{k+1}             */
        Pf1[c] = (Pf - dtau_pf * (divqD[c] + bd * (-(al / B) * Pfo - al * (Pt - Pto)) / dt - cc * Pt)) /
                 (1.0 + dtau_pf * (bd * al / (B * dt) + cc));
      }
}

/* ------------------------------------------ step 5: Maxwell stresses, Eq. 21 (backward Euler)
 * tau = (tau_o xi + 2 mu (edot + beta_n divVn delta_ij)) / (1 + xi),  xi = mu / (G dtS), with
 * dtS the stress sub-step of the appendix two-phase script;
 * on edges mu and xi are the means of the 4 surrounding centres; boundary-edge shear
 * stresses are zero (free slip). With a background shear stress (Eqs. 32-33) the xy strain
 * rate gains tau_bg / (2 mu0) at every xy-edge; on the wall edges the unknown velocity's part
 * is zero and mu, xi are the means over the centres next to the edge. */
void or_stress(const or_params *p, double dtS, const double *Vx, const double *Vy, const double *Vz,
               const double *divV, const double *divVn, const double *mu,
               const double *txxo, const double *tyyo, const double *tzzo,
               const double *txyo, const double *txzo, const double *tyzo,
               double *txx, double *tyy, double *tzz, double *txy, double *txz, double *tyz) {
  const double dx = h_x(p), dy = h_y(p), dz = h_z(p);
  const double Gdt = p->G * dtS, bn = p->beta_n;
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double m = mu[c], xi = m / Gdt, dv = divV[c];
        const double exx = (Vx[FX_(i + 1, j, k)] - Vx[FX_(i, j, k)]) / dx - dv / 3.0;
        const double eyy = (Vy[FY_(i, j + 1, k)] - Vy[FY_(i, j, k)]) / dy - dv / 3.0;
        const double ezz = (Vz[FZ_(i, j, k + 1)] - Vz[FZ_(i, j, k)]) / dz - dv / 3.0;
        txx[c] = (txxo[c] * xi + 2.0 * m * (exx + bn * divVn[c])) / (1.0 + xi);
        tyy[c] = (tyyo[c] * xi + 2.0 * m * (eyy + bn * divVn[c])) / (1.0 + xi);
        tzz[c] = (tzzo[c] * xi + 2.0 * m * (ezz + bn * divVn[c])) / (1.0 + xi);
      }
  const double ebg = 0.5 * p->tau_bg / p->mu0;   /* background xy strain rate */
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j <= NY; ++j)
      for (int i = 0; i <= NX; ++i) {
        double t = 0.0;
        if (i > 0 && i < NX && j > 0 && j < NY) {
          const double m = 0.25 * (mu[C_(i - 1, j - 1, k)] + mu[C_(i, j - 1, k)] +
                                   mu[C_(i - 1, j, k)] + mu[C_(i, j, k)]);
          const double xi = 0.25 * (mu[C_(i - 1, j - 1, k)] / Gdt + mu[C_(i, j - 1, k)] / Gdt +
                                    mu[C_(i - 1, j, k)] / Gdt + mu[C_(i, j, k)] / Gdt);
          const double e = 0.5 * ((Vx[FX_(i, j, k)] - Vx[FX_(i, j - 1, k)]) / dy +
                                  (Vy[FY_(i, j, k)] - Vy[FY_(i - 1, j, k)]) / dx) + ebg;
          t = (txyo[EXY_(i, j, k)] * xi + 2.0 * m * e) / (1.0 + xi);
        } else if (p->tau_bg != 0.0) {
          /* wall edge: the mean mu over the (two, or at a corner one) centres next to it */
          double msum = 0.0;
          int cnt = 0;
          for (int dj = -1; dj <= 0; ++dj)
            for (int di = -1; di <= 0; ++di)
              if (i + di >= 0 && i + di < NX && j + dj >= 0 && j + dj < NY) {
                msum += mu[C_(i + di, j + dj, k)];
                cnt += 1;
              }
          const double m = msum / cnt, xi = m / Gdt;
          t = (txyo[EXY_(i, j, k)] * xi + 2.0 * m * ebg) / (1.0 + xi);
        }
        txy[EXY_(i, j, k)] = t;
      }
#pragma omp parallel for
  for (int k = 0; k <= NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i <= NX; ++i) {
        double t = 0.0;
        if (i > 0 && i < NX && k > 0 && k < NZ) {
          const double m = 0.25 * (mu[C_(i - 1, j, k - 1)] + mu[C_(i, j, k - 1)] +
                                   mu[C_(i - 1, j, k)] + mu[C_(i, j, k)]);
          const double xi = 0.25 * (mu[C_(i - 1, j, k - 1)] / Gdt + mu[C_(i, j, k - 1)] / Gdt +
                                    mu[C_(i - 1, j, k)] / Gdt + mu[C_(i, j, k)] / Gdt);
          const double e = 0.5 * ((Vx[FX_(i, j, k)] - Vx[FX_(i, j, k - 1)]) / dz +
                                  (Vz[FZ_(i, j, k)] - Vz[FZ_(i - 1, j, k)]) / dx);
          t = (txzo[EXZ_(i, j, k)] * xi + 2.0 * m * e) / (1.0 + xi);
        }
        txz[EXZ_(i, j, k)] = t;
      }
#pragma omp parallel for
  for (int k = 0; k <= NZ; ++k)
    for (int j = 0; j <= NY; ++j)
      for (int i = 0; i < NX; ++i) {
        double t = 0.0;
        if (j > 0 && j < NY && k > 0 && k < NZ) {
          const double m = 0.25 * (mu[C_(i, j - 1, k - 1)] + mu[C_(i, j, k - 1)] +
                                   mu[C_(i, j - 1, k)] + mu[C_(i, j, k)]);
          const double xi = 0.25 * (mu[C_(i, j - 1, k - 1)] / Gdt + mu[C_(i, j, k - 1)] / Gdt +
                                    mu[C_(i, j - 1, k)] / Gdt + mu[C_(i, j, k)] / Gdt);
          const double e = 0.5 * ((Vy[FY_(i, j, k)] - Vy[FY_(i, j, k - 1)]) / dz +
                                  (Vz[FZ_(i, j, k)] - Vz[FZ_(i, j - 1, k)]) / dy);
          t = (tyzo[EYZ_(i, j, k)] * xi + 2.0 * m * e) / (1.0 + xi);
        }
        tyz[EYZ_(i, j, k)] = t;
      }
}

/* -------------------------------- step 6: momentum balance, Eq. 19 (interior faces only)
 * F_i = d_j tau_ij - d_i Pt - delta_iz (rho - rho_BG) g; zero on boundary faces. */
void or_momentum(const or_params *p, const double *txx, const double *tyy, const double *tzz,
                 const double *txy, const double *txz, const double *tyz,
                 const double *Pt, const double *rog, double *Fx, double *Fy, double *Fz) {
  const double dx = h_x(p), dy = h_y(p), dz = h_z(p);
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i <= NX; ++i) {
        double f = 0.0;
        if (i > 0 && i < NX)
          f = (txx[C_(i, j, k)] - txx[C_(i - 1, j, k)]) / dx +
              (txy[EXY_(i, j + 1, k)] - txy[EXY_(i, j, k)]) / dy +
              (txz[EXZ_(i, j, k + 1)] - txz[EXZ_(i, j, k)]) / dz -
              (Pt[C_(i, j, k)] - Pt[C_(i - 1, j, k)]) / dx;
        Fx[FX_(i, j, k)] = f;
      }
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j <= NY; ++j)
      for (int i = 0; i < NX; ++i) {
        double f = 0.0;
        if (j > 0 && j < NY)
          f = (txy[EXY_(i + 1, j, k)] - txy[EXY_(i, j, k)]) / dx +
              (tyy[C_(i, j, k)] - tyy[C_(i, j - 1, k)]) / dy +
              (tyz[EYZ_(i, j, k + 1)] - tyz[EYZ_(i, j, k)]) / dz -
              (Pt[C_(i, j, k)] - Pt[C_(i, j - 1, k)]) / dy;
        Fy[FY_(i, j, k)] = f;
      }
#pragma omp parallel for
  for (int k = 0; k <= NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        double f = 0.0;
        if (k > 0 && k < NZ)
          f = (txz[EXZ_(i + 1, j, k)] - txz[EXZ_(i, j, k)]) / dx +
              (tyz[EYZ_(i, j + 1, k)] - tyz[EYZ_(i, j, k)]) / dy +
              (tzz[C_(i, j, k)] - tzz[C_(i, j, k - 1)]) / dz -
              (Pt[C_(i, j, k)] - Pt[C_(i, j, k - 1)]) / dz -
              0.5 * (rog[C_(i, j, k - 1)] + rog[C_(i, j, k)]);
        Fz[FZ_(i, j, k)] = f;
      }
}

/* ------------------------------------------- step 7a: advection term of Eq. 22, log form
 * V . grad log(1 - phi) = V . grad(1 - phi) / (1 - phi): face velocity times the centred
 * face difference of (1 - phi), averaged over the two faces of each direction, divided by
 * (1 - phi) at the centre. Boundary faces carry no velocity (free slip) and add nothing. */
void or_advection(const or_params *p, const double *Vx, const double *Vy, const double *Vz,
                  const double *phi, double *adv) {
  const double dx = h_x(p), dy = h_y(p), dz = h_z(p);
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double omc = 1.0 - phi[c];
        double ax = 0.0, ay = 0.0, az = 0.0;
        if (i > 0) ax += Vx[FX_(i, j, k)] * (omc - (1.0 - phi[C_(i - 1, j, k)])) / dx;
        if (i < NX - 1) ax += Vx[FX_(i + 1, j, k)] * ((1.0 - phi[C_(i + 1, j, k)]) - omc) / dx;
        if (j > 0) ay += Vy[FY_(i, j, k)] * (omc - (1.0 - phi[C_(i, j - 1, k)])) / dy;
        if (j < NY - 1) ay += Vy[FY_(i, j + 1, k)] * ((1.0 - phi[C_(i, j + 1, k)]) - omc) / dy;
        if (k > 0) az += Vz[FZ_(i, j, k)] * (omc - (1.0 - phi[C_(i, j, k - 1)])) / dz;
        if (k < NZ - 1) az += Vz[FZ_(i, j, k + 1)] * ((1.0 - phi[C_(i, j, k + 1)]) - omc) / dz;
        adv[c] = 0.5 * (ax + ay + az) / omc;
      }
}

/* log(1 - phi) target of Eq. 22 after one backward-Euler step:
 * L = Lo - dt [beta_phi ((Pf - Pfo) - (Pt - Pto)) / dt + (Pf - Pt) / eta + V . grad L] */
static double porosity_log_target(const or_params *p, double Lo, double Pt, double Pf, double Pto,
                                  double Pfo, double eta, double adv) {
  const double comp = p->compaction_on ? (Pf - Pt) / eta : 0.0;
  return Lo - p->dt * (p->beta_phi * ((Pf - Pfo) - (Pt - Pto)) / p->dt + comp + adv);
}

/* ------------------------------ second stress invariant at centres (edge stresses averaged)
 * tau_II = sqrt(1/2 (txx^2 + tyy^2 + tzz^2) + <txy>^2 + <txz>^2 + <tyz>^2) */
void or_tau_II(const or_params *p, const double *txx, const double *tyy, const double *tzz,
               const double *txy, const double *txz, const double *tyz, double *tII) {
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double axy = 0.25 * (txy[EXY_(i, j, k)] + txy[EXY_(i + 1, j, k)] +
                                   txy[EXY_(i, j + 1, k)] + txy[EXY_(i + 1, j + 1, k)]);
        const double axz = 0.25 * (txz[EXZ_(i, j, k)] + txz[EXZ_(i + 1, j, k)] +
                                   txz[EXZ_(i, j, k + 1)] + txz[EXZ_(i + 1, j, k + 1)]);
        const double ayz = 0.25 * (tyz[EYZ_(i, j, k)] + tyz[EYZ_(i, j + 1, k)] +
                                   tyz[EYZ_(i, j, k + 1)] + tyz[EYZ_(i, j + 1, k + 1)]);
        tII[c] = sqrt(0.5 * (txx[c] * txx[c] + tyy[c] * tyy[c] + tzz[c] * tzz[c]) +
                      axy * axy + axz * axz + ayz * ayz);
      }
}

/* power-law shear viscosity target, Eq. 24 (weakening acts on the bulk viscosity, Eq. 26) */
static double mu_target(const or_params *p, double tII) {
  if (!p->powerlaw_on) return p->mu0;
  return p->mu0 / (1.0 + pow(tII / p->tau0, p->n_pow - 1.0));
}
/* bulk viscosity target, Eqs. 25-26: eta0 mu / phi, times R_weak where Pf > Pt */
static double eta_target(const or_params *p, double mu, double phi, double Pt, double Pf) {
  const double R = (Pf > Pt) ? p->R_weak : 1.0;
  return p->eta0 * mu / phi * R;
}

/* ------------------------------------------------------------------- scratch storage */
typedef struct {
  double *perm, *rog, *qx, *qy, *qz, *divqD, *divV, *divVn, *Pt1, *Pf1, *phi1, *adv;
  double *txx, *tyy, *tzz, *txy, *txz, *tyz, *Fx, *Fy, *Fz, *tII, *rpf;
} scratch;

static void scratch_free(scratch *w) {
  double **a = (double **)w;
  for (size_t n = 0; n < sizeof(scratch) / sizeof(double *); ++n) free(a[n]);
  memset(w, 0, sizeof *w);
}
static int scratch_alloc(const or_params *p, scratch *w) {
  memset(w, 0, sizeof *w);
  const long nc = n_centre(p);
  w->perm = calloc(nc, 8); w->rog = calloc(nc, 8); w->divqD = calloc(nc, 8);
  w->divV = calloc(nc, 8); w->divVn = calloc(nc, 8); w->Pt1 = calloc(nc, 8);
  w->Pf1 = calloc(nc, 8); w->phi1 = calloc(nc, 8); w->adv = calloc(nc, 8);
  w->txx = calloc(nc, 8); w->tyy = calloc(nc, 8); w->tzz = calloc(nc, 8); w->tII = calloc(nc, 8);
  w->rpf = calloc(nc, 8);
  w->qx = calloc(n_fx(p), 8); w->qy = calloc(n_fy(p), 8); w->qz = calloc(n_fz(p), 8);
  w->Fx = calloc(n_fx(p), 8); w->Fy = calloc(n_fy(p), 8); w->Fz = calloc(n_fz(p), 8);
  w->txy = calloc(n_exy(p), 8); w->txz = calloc(n_exz(p), 8); w->tyz = calloc(n_eyz(p), 8);
  double **a = (double **)w;
  for (size_t n = 0; n < sizeof(scratch) / sizeof(double *); ++n)
    if (!a[n]) { scratch_free(w); return OR_EINVAL; }
  return OR_OK;
}

/* ------------------------------------------------------------------- state helpers */
int or_init_viscosities(const or_params *p, or_state *s) {
  if (!params_ok(p) || !s) return OR_EINVAL;
  const long nc = n_centre(p);
  for (long c = 0; c < nc; ++c) {
    s->mu[c] = p->mu0;
    s->eta[c] = p->eta0 * s->mu[c] / s->phi[c];
  }
  return OR_OK;
}

int or_begin_step(const or_params *p, or_state *s) {
  if (!params_ok(p) || !s) return OR_EINVAL;
  const long nc = n_centre(p);
  double mu_max = 0.0;
  for (long c = 0; c < nc; ++c) {
    s->Pto[c] = s->Pt[c];
    s->Pfo[c] = s->Pf[c];
    s->Lo[c] = log(1.0 - s->phi[c]);
    mu_max = fmax(mu_max, s->mu[c]);
  }
  /* stress sub-step: the largest xi = mu / (G dtS) equals xsi_w */
  s->dtS = mu_max / (p->G * p->xsi_w);
  if (s->nsteps == 0 || s->dt_cum >= s->dtS) {
    for (long c = 0; c < nc; ++c) {
      s->txxo[c] = s->txx[c];
      s->tyyo[c] = s->tyy[c];
      s->tzzo[c] = s->tzz[c];
    }
    memcpy(s->txyo, s->txy, n_exy(p) * sizeof(double));
    memcpy(s->txzo, s->txz, n_exz(p) * sizeof(double));
    memcpy(s->tyzo, s->tyz, n_eyz(p) * sizeof(double));
    s->dt_cum = 0.0;
  }
  s->nsteps += 1;
  return OR_OK;
}

static double max_abs(const double *a, long n, int *bad) {
  double m = 0.0;
  int nonfinite = 0;
#pragma omp parallel for reduction(max : m) reduction(| : nonfinite)
  for (long c = 0; c < n; ++c) {
    const double v = fabs(a[c]);
    if (!isfinite(v)) nonfinite |= 1;
    else if (v > m) m = v;
  }
  *bad |= nonfinite;
  return m;
}

/* One PT iteration k -> k+1 in the order of the file header. */
static int iteration_impl(const or_params *p, or_state *s, int it, scratch *w, or_res *res,
                          int *checked) {
  const long nc = n_centre(p);
  const int do_picard = (it % p->nup) == 0;

  or_coefficients(p, s->phi, s->logk, w->perm, w->rog);                        /* 1 */
  or_darcy(p, s->Pf, w->perm, w->qx, w->qy, w->qz, w->divqD);                  /* 2 */
  or_divergence(p, s->Vx, s->Vy, s->Vz, s->Pt, s->Pf, s->Pto, s->Pfo, s->phi,   /* 3 */
                s->eta, w->divV, w->divVn);
  pressure_update(p, s, w->perm, w->divV, w->divqD, w->Pt1, w->Pf1);           /* 4 */
  if (do_picard) {          /* fluid-pressure residual of iterate k, for the norms of step 10 */
#pragma omp parallel for
    for (long c = 0; c < nc; ++c)
      w->rpf[c] = pf_residual(p, w->divqD[c], s->Pt[c], s->Pf[c], s->Pto[c], s->Pfo[c],
                              s->eta[c], s->phi[c]);
  }
  or_stress(p, s->dtS, s->Vx, s->Vy, s->Vz, w->divV, w->divVn, s->mu,          /* 5 */
            s->txxo, s->tyyo, s->tzzo, s->txyo, s->txzo, s->tyzo,
            w->txx, w->tyy, w->tzz, w->txy, w->txz, w->tyz);
  if (p->mech_on) {                                                             /* 6 */
    or_momentum(p, w->txx, w->tyy, w->tzz, w->txy, w->txz, w->tyz, w->Pt1, w->rog,
                w->Fx, w->Fy, w->Fz);
  } else {
    memset(w->Fx, 0, n_fx(p) * 8); memset(w->Fy, 0, n_fy(p) * 8); memset(w->Fz, 0, n_fz(p) * 8);
  }
  or_advection(p, s->Vx, s->Vy, s->Vz, s->phi, w->adv);                        /* 7 */
#pragma omp parallel for
  for (long c = 0; c < nc; ++c) {
    const double L1 = porosity_log_target(p, s->Lo[c], w->Pt1[c], w->Pf1[c], s->Pto[c],
                                          s->Pfo[c], s->eta[c], w->adv[c]);
    w->phi1[c] = 1.0 - exp(L1);
  }
  if (p->mech_on) {                                                             /* 6 + 8 */
#pragma omp parallel for
    for (int k = 0; k < NZ; ++k)
      for (int j = 0; j < NY; ++j)
        for (int i = 1; i < NX; ++i) {
          const long f = FX_(i, j, k);
          s->Rx[f] = w->Fx[f] / p->rho_i + p->damp_x * s->Rx[f];
          const double dtau = 0.5 * (dtau_v(p, s->mu[C_(i - 1, j, k)]) + dtau_v(p, s->mu[C_(i, j, k)]));
          s->Vx[f] += dtau * s->Rx[f];
        }
#pragma omp parallel for
    for (int k = 0; k < NZ; ++k)
      for (int j = 1; j < NY; ++j)
        for (int i = 0; i < NX; ++i) {
          const long f = FY_(i, j, k);
          s->Ry[f] = w->Fy[f] / p->rho_i + p->damp_y * s->Ry[f];
          const double dtau = 0.5 * (dtau_v(p, s->mu[C_(i, j - 1, k)]) + dtau_v(p, s->mu[C_(i, j, k)]));
          s->Vy[f] += dtau * s->Ry[f];
        }
#pragma omp parallel for
    for (int k = 1; k < NZ; ++k)
      for (int j = 0; j < NY; ++j)
        for (int i = 0; i < NX; ++i) {
          const long f = FZ_(i, j, k);
          s->Rz[f] = w->Fz[f] / p->rho_i + p->damp_z * s->Rz[f];
          const double dtau = 0.5 * (dtau_v(p, s->mu[C_(i, j, k - 1)]) + dtau_v(p, s->mu[C_(i, j, k)]));
          s->Vz[f] += dtau * s->Rz[f];
        }
  }

  double r_pic = 0.0;
  int bad = 0;
  if (do_picard) {                                                              /* 9 */
    or_tau_II(p, w->txx, w->tyy, w->tzz, w->txy, w->txz, w->tyz, w->tII);
    double m = 0.0;
    int nonfinite = 0;
#pragma omp parallel for reduction(max : m) reduction(| : nonfinite)
    for (long c = 0; c < nc; ++c) {
      const double mus = mu_target(p, w->tII[c]);
      const double mu_old = s->mu[c], eta_old = s->eta[c];
      const double mu_new = exp(p->rel_mu * log(mus) + (1.0 - p->rel_mu) * log(mu_old));
      const double etas = eta_target(p, mu_new, w->phi1[c], w->Pt1[c], w->Pf1[c]);
      const double eta_new = exp(p->rel_eta * log(etas) + (1.0 - p->rel_eta) * log(eta_old));
      const double d = fmax(fabs(log(mus) - log(mu_old)), fabs(log(etas) - log(eta_old)));
      if (!isfinite(d)) nonfinite |= 1;
      else if (d > m) m = d;
      s->mu[c] = mu_new;
      s->eta[c] = eta_new;
    }
    r_pic = m;
    bad |= nonfinite;
  }
  if (do_picard) {                                                              /* 10 */
    res->r_v = fmax(max_abs(w->Fx, n_fx(p), &bad),
                    fmax(max_abs(w->Fy, n_fy(p), &bad), max_abs(w->Fz, n_fz(p), &bad)));
    res->r_pt = max_abs(w->divVn, nc, &bad);
    res->r_pf = max_abs(w->rpf, nc, &bad);
    res->r_pic = r_pic;
    if (checked) *checked = 1;
  } else if (checked) {
    *checked = 0;
  }
  /* commit iterate k+1 of the centre fields */
  memcpy(s->Pt, w->Pt1, nc * 8);
  memcpy(s->Pf, w->Pf1, nc * 8);
  memcpy(s->phi, w->phi1, nc * 8);
  return bad ? OR_ENAN : OR_OK;
}

int or_iteration(const or_params *p, or_state *s, int it, or_res *res, int *checked) {
  if (!params_ok(p) || !s || !res || it < 1) return OR_EINVAL;
  scratch w;
  if (scratch_alloc(p, &w) != OR_OK) return OR_EINVAL;
  const int rc = iteration_impl(p, s, it, &w, res, checked);
  scratch_free(&w);
  return rc;
}

int or_end_step(const or_params *p, or_state *s) {
  if (!params_ok(p) || !s) return OR_EINVAL;
  scratch w;
  if (scratch_alloc(p, &w) != OR_OK) return OR_EINVAL;
  or_divergence(p, s->Vx, s->Vy, s->Vz, s->Pt, s->Pf, s->Pto, s->Pfo, s->phi, s->eta,
                w.divV, w.divVn);
  or_stress(p, s->dtS, s->Vx, s->Vy, s->Vz, w.divV, w.divVn, s->mu, s->txxo, s->tyyo, s->tzzo,
            s->txyo, s->txzo, s->tyzo, s->txx, s->tyy, s->tzz, s->txy, s->txz, s->tyz);
  scratch_free(&w);
  s->dt_cum += p->dt;
  return OR_OK;
}

int or_iterate_n(const or_params *p, or_state *s, int it0, int niter, or_res *res) {
  if (!params_ok(p) || !s || !res || it0 < 0 || niter < 0) return OR_EINVAL;
  scratch w;
  if (scratch_alloc(p, &w) != OR_OK) return OR_EINVAL;
  int rc = OR_OK, checked = 0;
  for (int n = 1; n <= niter && rc == OR_OK; ++n) rc = iteration_impl(p, s, it0 + n, &w, res, &checked);
  scratch_free(&w);
  return rc;
}

int or_step(const or_params *p, or_state *s, int *iters, or_res *res) {
  if (!params_ok(p) || !s || !res) return OR_EINVAL;
  int rc = or_begin_step(p, s);
  if (rc != OR_OK) return rc;
  scratch w;
  if (scratch_alloc(p, &w) != OR_OK) return OR_EINVAL;
  int it = 0, converged = 0;
  memset(res, 0, sizeof *res);
  while (it < p->max_iter) {
    ++it;
    int checked = 0;
    rc = iteration_impl(p, s, it, &w, res, &checked);
    if (rc != OR_OK) break;
    if (checked && fmax(fmax(res->r_v, res->r_pt), fmax(res->r_pf, res->r_pic)) < p->tol) {
      converged = 1;
      break;
    }
  }
  scratch_free(&w);
  if (iters) *iters = it;
  if (rc != OR_OK) return rc;
  rc = or_end_step(p, s);
  if (rc != OR_OK) return rc;
  return converged ? OR_OK : OR_ENOTCONV;
}

int or_system_residual(const or_params *p, const or_state *s,
                       double *out_Vx, double *out_Vy, double *out_Vz, double *out_pt,
                       double *out_pf, double *out_L, double *out_mu, double *out_eta) {
  if (!params_ok(p) || !s) return OR_EINVAL;
  scratch w;
  if (scratch_alloc(p, &w) != OR_OK) return OR_EINVAL;
  const long nc = n_centre(p);
  or_coefficients(p, s->phi, s->logk, w.perm, w.rog);
  or_darcy(p, s->Pf, w.perm, w.qx, w.qy, w.qz, w.divqD);
  or_divergence(p, s->Vx, s->Vy, s->Vz, s->Pt, s->Pf, s->Pto, s->Pfo, s->phi, s->eta,
                w.divV, w.divVn);
  or_stress(p, s->dtS, s->Vx, s->Vy, s->Vz, w.divV, w.divVn, s->mu, s->txxo, s->tyyo, s->tzzo,
            s->txyo, s->txzo, s->tyzo, w.txx, w.tyy, w.tzz, w.txy, w.txz, w.tyz);
  or_momentum(p, w.txx, w.tyy, w.tzz, w.txy, w.txz, w.tyz, s->Pt, w.rog, out_Vx, out_Vy, out_Vz);
  or_advection(p, s->Vx, s->Vy, s->Vz, s->phi, w.adv);
  or_tau_II(p, w.txx, w.tyy, w.tzz, w.txy, w.txz, w.tyz, w.tII);
  for (long c = 0; c < nc; ++c) {
    out_pt[c] = w.divVn[c];
    out_pf[c] = pf_residual(p, w.divqD[c], s->Pt[c], s->Pf[c], s->Pto[c], s->Pfo[c], s->eta[c],
                            s->phi[c]);
    out_L[c] = log(1.0 - s->phi[c]) -
               porosity_log_target(p, s->Lo[c], s->Pt[c], s->Pf[c], s->Pto[c], s->Pfo[c],
                                   s->eta[c], w.adv[c]);
    out_mu[c] = log(s->mu[c]) - log(mu_target(p, w.tII[c]));
    out_eta[c] = log(s->eta[c]) - log(eta_target(p, s->mu[c], s->phi[c], s->Pt[c], s->Pf[c]));
  }
  scratch_free(&w);
  return OR_OK;
}

int or_max_threads(void) { return omp_get_max_threads(); }
