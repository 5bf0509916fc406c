/* rx_oracle.c — plain FP64 CPU oracle of the reactive porosity-wave solver (thesis Art. 3,
 * Eqs. 8-10, as discretised by its appendix A.6 script). TEST INFRASTRUCTURE ONLY: used by
 * tests/ and bench.py's CPU baseline leg; the CUDA path never links it and shares no code.
 *
 * Unknowns at the centres of a cell-centred nx x ny x nz grid (dx = lx / nx): fluid pressure
 * Pf (effective pressure Pe = -Pf), porosity phi, mass fraction of volatiles bound to the
 * solid Xs, and the pseudo-transient rate R that the fluid-pressure update relaxes towards.
 * One implicit physical step of length dt is iterated to its fixed point; one PT iteration
 * from the iterate (Pf, phi, Xs) and the old step (Pf_o, phi_o, Xs_o) computes, per cell:
 *   Xseq  = clamp(beta_x Pf + Xs_max / 2, 0, Xs_max)                      (Eq. 4 reading)
 *   dXs   = (Xseq - Xs) / tau                                             (Eq. 10)
 *   R     = (-div qD + Pe / (eta (1 - phi)) + S_r (1 - phi)(1 + dX)/(1 - Xs) dXs) / BP  (Eq. 8)
 *   Xs'   = (Xs_o + (dt / tau) Xseq) / (1 + dt / tau)           (backward Euler, local-implicit)
 *   Pf'   = Pf + dtau (R - (Pf - Pf_o) / dt) / (1 + dtau (1 / dt + a))   (pseudo-transient)
 *   dphi  = (1 - phi) (Bphi R - Pe / (eta (1 - phi)) - (1 + dX) / (1 - Xs) dXs)   (Eq. 9)
 *   phi'  = clamp(phi_o + dt dphi, 1e-4, 1)
 * with Pe = -Pf, BP = phi beta_f + beta_d - (1 + phi) beta_s, Bphi = beta_d - beta_s / (1 - phi),
 * S_r = 1 - rho_s / (rho_f (1 + dX)), a = -dR/dPf of the cell's own terms (compaction and the
 * reaction source through Xseq; the local diagonal, taken implicitly), and the Darcy flux
 * qD = -k (grad Pf - rho_f g e_z), k = k0 (phi / phi0)^3 averaged arithmetically to the faces,
 * zero through the walls. Every right-hand side is evaluated at the iterate (Jacobi); R is the
 * rate dPf/dt the fixed point satisfies and is kept as an output. The pseudo step
 * dtau = min(dx, dy, dz)^2 / max(k / BP) / cfl_div is taken at the start of the step and after
 * every nup-th iteration from the porosity then current; at those iterations the change
 * max(|phi' - phi|, |Pf' - Pf| / pf_scale, |Xs' - Xs|) is compared with tol.
 */
#include "rx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NX (p->nx)
#define NY (p->ny)
#define NZ (p->nz)
#define C_(i, j, k) ((long)(i) + (long)NX * ((long)(j) + (long)NY * (long)(k)))

static long n_cells(const rx_params *p) { return (long)NX * NY * NZ; }

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

double rx_perm(const rx_params *p, double phi) {
  const double r = phi / p->phi0;
  return p->k0 * r * r * r;
}

double rx_beta_p(const rx_params *p, double phi) {
  return phi * p->beta_f + p->beta_d - (1.0 + phi) * p->beta_s;
}

double rx_xseq(const rx_params *p, double Pf) {
  return clampd(p->beta_x * Pf + 0.5 * p->xs_max, 0.0, p->xs_max);
}

/* div qD at every cell, qD = -k_face (dPf/dn - rho_f g [z faces]), zero through the walls. */
void rx_div_qd(const rx_params *p, const double *Pf, const double *phi, double *divq) {
  const double dx = p->lx / NX, dy = p->ly / NY, dz = p->lz / NZ;
#pragma omp parallel for
  for (int k = 0; k < NZ; ++k)
    for (int j = 0; j < NY; ++j)
      for (int i = 0; i < NX; ++i) {
        const long c = C_(i, j, k);
        const double kc = rx_perm(p, phi[c]);
        double qxl = 0.0, qxr = 0.0, qyl = 0.0, qyr = 0.0, qzl = 0.0, qzr = 0.0;
        if (i > 0) qxl = -0.5 * (rx_perm(p, phi[C_(i - 1, j, k)]) + kc) * (Pf[c] - Pf[C_(i - 1, j, k)]) / dx;
        if (i < NX - 1) qxr = -0.5 * (kc + rx_perm(p, phi[C_(i + 1, j, k)])) * (Pf[C_(i + 1, j, k)] - Pf[c]) / dx;
        if (j > 0) qyl = -0.5 * (rx_perm(p, phi[C_(i, j - 1, k)]) + kc) * (Pf[c] - Pf[C_(i, j - 1, k)]) / dy;
        if (j < NY - 1) qyr = -0.5 * (kc + rx_perm(p, phi[C_(i, j + 1, k)])) * (Pf[C_(i, j + 1, k)] - Pf[c]) / dy;
        if (k > 0)
          qzl = -0.5 * (rx_perm(p, phi[C_(i, j, k - 1)]) + kc) * ((Pf[c] - Pf[C_(i, j, k - 1)]) / dz - p->rhof * p->g);
        if (k < NZ - 1)
          qzr = -0.5 * (kc + rx_perm(p, phi[C_(i, j, k + 1)])) * ((Pf[C_(i, j, k + 1)] - Pf[c]) / dz - p->rhof * p->g);
        divq[c] = (qxr - qxl) / dx + (qyr - qyl) / dy + (qzr - qzl) / dz;
      }
}

double rx_pseudo_step(const rx_params *p, const double *phi) {
  const double dx = p->lx / NX, dy = p->ly / NY, dz = p->lz / NZ;
  const double h = fmin(dx, fmin(dy, dz));
  double m = 0.0;
  for (long c = 0; c < n_cells(p); ++c) m = fmax(m, rx_perm(p, phi[c]) / rx_beta_p(p, phi[c]));
  return h * h / m / p->cfl_div;
}

int rx_begin_step(const rx_params *p, rx_state *s) {
  const long n = n_cells(p);
  memcpy(s->Pf_o, s->Pf, n * sizeof(double));
  memcpy(s->phi_o, s->phi, n * sizeof(double));
  memcpy(s->Xs_o, s->Xs, n * sizeof(double));
  s->dtau = rx_pseudo_step(p, s->phi);
  return RX_OK;
}

int rx_iteration(const rx_params *p, rx_state *s, int it, double *change) {
  const long n = n_cells(p);
  double *divq = malloc(n * sizeof(double));
  double *Pf1 = malloc(n * sizeof(double)), *phi1 = malloc(n * sizeof(double));
  double *Xs1 = malloc(n * sizeof(double)), *R1 = malloc(n * sizeof(double));
  if (!divq || !Pf1 || !phi1 || !Xs1 || !R1) {
    free(divq); free(Pf1); free(phi1); free(Xs1); free(R1);
    return RX_EINVAL;
  }
  rx_div_qd(p, s->Pf, s->phi, divq);
  const double Sr = 1.0 - p->rhos / (p->rhof * (1.0 + p->dX));
  double err = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : err) reduction(| : bad)
  for (long c = 0; c < n; ++c) {
    const double Pf = s->Pf[c], phi = s->phi[c], Xs = s->Xs[c];
    const double Pe = -Pf;
    const double xr = p->beta_x * Pf + 0.5 * p->xs_max;
    const double xseq = clampd(xr, 0.0, p->xs_max);
    const double dXs = (xseq - Xs) / p->tau;
    const double bp = rx_beta_p(p, phi);
    const double src = Sr * (1.0 - phi) * (1.0 + p->dX) / (1.0 - Xs);
    const double R = (-divq[c] + Pe / (p->eta * (1.0 - phi)) + src * dXs) / bp;
    /* -dR/dPf of the cell's own terms; Xseq depends on Pf only between its clamps */
    const double dxs_dpf = (xr > 0.0 && xr < p->xs_max) ? p->beta_x : 0.0;
    const double a = (1.0 / (p->eta * (1.0 - phi)) - src * dxs_dpf / p->tau) / bp;
    Xs1[c] = (s->Xs_o[c] + p->dt / p->tau * xseq) / (1.0 + p->dt / p->tau);
    Pf1[c] = Pf + s->dtau * (R - (Pf - s->Pf_o[c]) / p->dt) / (1.0 + s->dtau * (1.0 / p->dt + a));
    const double Bphi = p->beta_d - p->beta_s / (1.0 - phi);
    const double dphi = (1.0 - phi) * (Bphi * R - Pe / (p->eta * (1.0 - phi)) - (1.0 + p->dX) / (1.0 - Xs) * dXs);
    phi1[c] = clampd(s->phi_o[c] + p->dt * dphi, 1e-4, 1.0);
    R1[c] = R;
    const double e = fmax(fabs(phi1[c] - phi), fmax(fabs(Pf1[c] - Pf) / p->pf_scale, fabs(Xs1[c] - Xs)));
    err = fmax(err, e);
    bad |= !(isfinite(Pf1[c]) && isfinite(phi1[c]) && isfinite(Xs1[c]));   /* fmax drops NaN */
  }
  if (bad) err = NAN;
  memcpy(s->Pf, Pf1, n * sizeof(double));
  memcpy(s->phi, phi1, n * sizeof(double));
  memcpy(s->Xs, Xs1, n * sizeof(double));
  memcpy(s->R, R1, n * sizeof(double));
  free(divq); free(Pf1); free(phi1); free(Xs1); free(R1);
  if (change) *change = err;
  if (!isfinite(err)) return RX_ENAN;
  if (it % p->nup == 0) s->dtau = rx_pseudo_step(p, s->phi);
  return RX_OK;
}

int rx_step(const rx_params *p, rx_state *s, int *iters, double *change) {
  rx_begin_step(p, s);
  double err = 0.0;
  int it = 0;
  while (it < p->max_iter) {
    ++it;
    const int rc = rx_iteration(p, s, it, &err);
    if (rc != RX_OK) {
      if (iters) *iters = it;
      if (change) *change = err;
      return rc;
    }
    if (it % p->nup == 0 && err < p->tol) break;
  }
  if (iters) *iters = it;
  if (change) *change = err;
  return (it % p->nup == 0 && err < p->tol) ? RX_OK : RX_ENOTCONV;
}

int rx_iterate_n(const rx_params *p, rx_state *s, int niter, double *change) {
  rx_begin_step(p, s);
  double err = 0.0;
  for (int it = 1; it <= niter; ++it) {
    const int rc = rx_iteration(p, s, it, &err);
    if (rc != RX_OK) return rc;
  }
  if (change) *change = err;
  return RX_OK;
}
