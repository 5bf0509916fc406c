/* rx_mg_oracle.c — plain FP64 CPU oracle of the geometric-multigrid acceleration of the reactive
 * porosity-wave step (thesis Art. 3, Eqs. 8-10 discretised as in rx_oracle.c; the thesis's
 * future-work section on multigrid-accelerated pseudo-transient iterations). TEST
 * INFRASTRUCTURE ONLY: used by tests/ and bench.py's CPU baseline leg; the CUDA path never
 * links it and shares no code.
 *
 * The thesis observes that its pseudo-transient (PT) iterations become Jacobi iterations when
 * the pseudo step is taken locally, weighted Jacobi when that local step is scaled by a weight,
 * and proposes geometric multigrid on top of them, with one of the standard treatments of the
 * nonlinearity. This oracle takes the full approximation scheme (FAS) V-cycle of the multigrid
 * textbook the thesis cites (Trottenberg, Oosterlee and Schueller), smoothing by the reactive
 * PT iteration itself with local pseudo steps, and cell-centred 2 x 2 x 2 coarsening.
 *
 * Step equations on a grid (cell-centred, spacing d; R, dphi, Xseq, BP, a as in rx_oracle.c),
 * written as "target - current":
 *   gP   = R(u) - (Pf - Pf_o) / dt + fP                               (Eq. 8, implicit step)
 *   gphi = clamp(phi_o + dt dphi(u), 1e-4, 1) + fphi - phi            (Eq. 9)
 *   gX   = (Xs_o + (dt / tau) Xseq(Pf)) / (1 + dt / tau) + fX - Xs    (Eq. 10, backward Euler)
 * with f = 0 on the finest grid and the FAS sources on the coarser ones.
 * Smoothing sweep (Jacobi: every right-hand side at the sweep's input):
 *   Pf' = Pf + gP / (Dk / (omega BP) + 1 / dt + a),  phi' = phi + gphi,  Xs' = Xs + gX,
 * Dk = sum over the cell's interior faces of the face permeability / d^2 (the diagonal of the
 * Darcy operator). This is the PT update of rx_oracle.c with the local pseudo step
 * dtau = omega BP / Dk in place of the global one: weighted Jacobi on the Darcy part, the
 * cell's own terms implicit.
 * Transfer: restriction = mean of the 8 children (state and residuals); prolongation =
 * trilinear interpolation of the coarse correction to the fine centres (weights 3/4 and 1/4
 * per direction), the neighbour index held at the wall (zero-gradient extrapolation); phi is
 * clamped to [1e-4, 1] after a correction.
 * FAS V-cycle on level l (l = 0 finest, levels - 1 coarsest):
 *   coarsest: nu_coarse sweeps;
 *   otherwise: nu_pre sweeps; r = g(u) (with f); u_c = Restrict(u); u0_c = u_c;
 *              f_c = Restrict(r) - g_c(u0_c) (g_c without f); V-cycle(l + 1);
 *              u += Prolong(u_c - u0_c); nu_post sweeps.
 * The old-step fields of a coarse level are the restriction of the finer level's, once per
 * physical step. A converged fine solution (g = 0) gives f_c = -g_c(u0_c), whose coarse solution
 * is u0_c itself: the correction vanishes, so the cycle's fixed point is the plain PT
 * iteration's. The change of a cycle is max(|dphi|, |dPf| / pf_scale, |dXs|) of its last sweep
 * on the finest grid; the rate R of that sweep is kept as the output R.
 */
#include "rx_mg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

static long idx3(int nx, int ny, int i, int j, int k) { return (long)i + (long)nx * ((long)j + (long)ny * (long)k); }

void rx_mg_restrict(int nx, int ny, int nz, const double *fine, double *coarse) {
  const int mx = nx / 2, my = ny / 2, mz = nz / 2;
#pragma omp parallel for
  for (int K = 0; K < mz; ++K)
    for (int J = 0; J < my; ++J)
      for (int I = 0; I < mx; ++I) {
        double s = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) s += fine[idx3(nx, ny, 2 * I + a, 2 * J + b, 2 * K + c)];
        coarse[idx3(mx, my, I, J, K)] = s / 8.0;
      }
}

/* the coarse neighbour on the child's side, held inside [0, m) */
static int side_nb(int i, int m) {
  const int I = i / 2;
  const int n = (i % 2) ? I + 1 : I - 1;
  return n < 0 ? 0 : (n > m - 1 ? m - 1 : n);
}

void rx_mg_prolong_add(int nx, int ny, int nz, const double *e, double *fine) {
  const int mx = nx / 2, my = ny / 2, mz = nz / 2;
#pragma omp parallel for
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const int Ix[2] = {i / 2, side_nb(i, mx)}, Jy[2] = {j / 2, side_nb(j, my)}, Kz[2] = {k / 2, side_nb(k, mz)};
        const double w[2] = {0.75, 0.25};
        double v = 0.0;
        for (int c = 0; c < 2; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) v += w[a] * w[b] * w[c] * e[idx3(mx, my, Ix[a], Jy[b], Kz[c])];
        fine[idx3(nx, ny, i, j, k)] += v;
      }
}

void rx_mg_equations(const rx_params *p, const double *Pf, const double *phi, const double *Xs,
                     const double *Pf_o, const double *phi_o, const double *Xs_o, const double *fP,
                     const double *fphi, const double *fX, double omega, double *gP, double *gphi,
                     double *gX, double *den, double *R) {
  const int nx = p->nx, ny = p->ny, nz = p->nz;
  const long n = (long)nx * ny * nz;
  double *divq = malloc(n * sizeof(double));
  if (!divq) return;
  rx_div_qd(p, Pf, phi, divq);
  const double dx = p->lx / nx, dy = p->ly / ny, dz = p->lz / nz;
  const double Sr = 1.0 - p->rhos / (p->rhof * (1.0 + p->dX));
#pragma omp parallel for
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long c = idx3(nx, ny, i, j, k);
        const double pf = Pf[c], ph = phi[c], xs = Xs[c];
        const double Pe = -pf;
        const double xr = p->beta_x * pf + 0.5 * p->xs_max;
        const double xseq = clampd(xr, 0.0, p->xs_max);
        const double dXs = (xseq - xs) / p->tau;
        const double bp = rx_beta_p(p, ph);
        const double src = Sr * (1.0 - ph) * (1.0 + p->dX) / (1.0 - xs);
        const double Rc = (-divq[c] + Pe / (p->eta * (1.0 - ph)) + src * dXs) / bp;
        const double dxs_dpf = (xr > 0.0 && xr < p->xs_max) ? p->beta_x : 0.0;
        const double a = (1.0 / (p->eta * (1.0 - ph)) - src * dxs_dpf / p->tau) / bp;
        /* diagonal of the Darcy operator: face permeability (arithmetic mean) over d^2 */
        const double kc = rx_perm(p, ph);
        double Dk = 0.0;
        if (i > 0) Dk += 0.5 * (rx_perm(p, phi[c - 1]) + kc) / (dx * dx);
        if (i < nx - 1) Dk += 0.5 * (kc + rx_perm(p, phi[c + 1])) / (dx * dx);
        if (j > 0) Dk += 0.5 * (rx_perm(p, phi[c - nx]) + kc) / (dy * dy);
        if (j < ny - 1) Dk += 0.5 * (kc + rx_perm(p, phi[c + nx])) / (dy * dy);
        if (k > 0) Dk += 0.5 * (rx_perm(p, phi[c - (long)nx * ny]) + kc) / (dz * dz);
        if (k < nz - 1) Dk += 0.5 * (kc + rx_perm(p, phi[c + (long)nx * ny])) / (dz * dz);
        const double bphi = p->beta_d - p->beta_s / (1.0 - ph);
        const double dphi = (1.0 - ph) * (bphi * Rc - Pe / (p->eta * (1.0 - ph)) - (1.0 + p->dX) / (1.0 - xs) * dXs);
        gP[c] = Rc - (pf - Pf_o[c]) / p->dt + (fP ? fP[c] : 0.0);
        den[c] = Dk / (omega * bp) + 1.0 / p->dt + a;
        gphi[c] = clampd(phi_o[c] + p->dt * dphi, 1e-4, 1.0) + (fphi ? fphi[c] : 0.0) - ph;
        gX[c] = (Xs_o[c] + p->dt / p->tau * xseq) / (1.0 + p->dt / p->tau) + (fX ? fX[c] : 0.0) - xs;
        R[c] = Rc;
      }
  free(divq);
}

typedef struct {
  rx_params p;                         /* this level's grid; physics and numerics as the finest */
  long n;
  double *Pf, *phi, *Xs, *Pf_o, *phi_o, *Xs_o;
  double *fP, *fphi, *fX;              /* FAS sources (NULL on the finest level) */
  double *Pf0, *phi0, *Xs0;            /* restricted state before the coarse solve */
  double *gP, *gphi, *gX, *den, *R;    /* equations of the current iterate */
} level;

#define LEVEL_OWNED 12   /* arrays a coarse level allocates: iterate, old, f, u0 (3 each) */
#define LEVEL_SCRATCH 4  /* gP, gphi, gX, den (R too on coarse levels) */

static double sweep(level *L, double omega) {
  rx_mg_equations(&L->p, L->Pf, L->phi, L->Xs, L->Pf_o, L->phi_o, L->Xs_o, L->fP, L->fphi, L->fX, omega, L->gP,
                  L->gphi, L->gX, L->den, L->R);
  double err = 0.0;
  int bad = 0;
#pragma omp parallel for reduction(max : err) reduction(| : bad)
  for (long c = 0; c < L->n; ++c) {
    const double dPf = L->gP[c] / L->den[c];
    L->Pf[c] += dPf;
    L->phi[c] += L->gphi[c];
    L->Xs[c] += L->gX[c];
    err = fmax(err, fmax(fabs(L->gphi[c]), fmax(fabs(dPf) / L->p.pf_scale, fabs(L->gX[c]))));
    bad |= !(isfinite(L->Pf[c]) && isfinite(L->phi[c]) && isfinite(L->Xs[c]));   /* fmax drops NaN */
  }
  return bad ? NAN : err;
}

static double vcycle(level *Ls, int l, const rx_mg_params *mg) {
  level *L = &Ls[l];
  double err = 0.0;
  if (l == mg->levels - 1) {
    for (int s = 0; s < mg->nu_coarse; ++s) err = sweep(L, mg->omega);
    return err;
  }
  for (int s = 0; s < mg->nu_pre; ++s) err = sweep(L, mg->omega);
  level *C = &Ls[l + 1];
  const int nx = L->p.nx, ny = L->p.ny, nz = L->p.nz;
  /* residual of the smoothed iterate, restricted with the iterate itself */
  rx_mg_equations(&L->p, L->Pf, L->phi, L->Xs, L->Pf_o, L->phi_o, L->Xs_o, L->fP, L->fphi, L->fX, mg->omega, L->gP,
                  L->gphi, L->gX, L->den, L->R);
  rx_mg_restrict(nx, ny, nz, L->Pf, C->Pf);
  rx_mg_restrict(nx, ny, nz, L->phi, C->phi);
  rx_mg_restrict(nx, ny, nz, L->Xs, C->Xs);
  memcpy(C->Pf0, C->Pf, C->n * sizeof(double));
  memcpy(C->phi0, C->phi, C->n * sizeof(double));
  memcpy(C->Xs0, C->Xs, C->n * sizeof(double));
  rx_mg_restrict(nx, ny, nz, L->gP, C->fP);
  rx_mg_restrict(nx, ny, nz, L->gphi, C->fphi);
  rx_mg_restrict(nx, ny, nz, L->gX, C->fX);
  /* FAS source: f_c = Restrict(r) - g_c(u0_c) */
  rx_mg_equations(&C->p, C->Pf0, C->phi0, C->Xs0, C->Pf_o, C->phi_o, C->Xs_o, NULL, NULL, NULL, mg->omega, C->gP,
                  C->gphi, C->gX, C->den, C->R);
  for (long c = 0; c < C->n; ++c) {
    C->fP[c] -= C->gP[c];
    C->fphi[c] -= C->gphi[c];
    C->fX[c] -= C->gX[c];
  }
  vcycle(Ls, l + 1, mg);
  /* coarse correction e = u_c - u0_c, interpolated and added */
  double *e = malloc(C->n * sizeof(double));
  if (!e) return NAN;
  for (long c = 0; c < C->n; ++c) e[c] = C->Pf[c] - C->Pf0[c];
  rx_mg_prolong_add(nx, ny, nz, e, L->Pf);
  for (long c = 0; c < C->n; ++c) e[c] = C->phi[c] - C->phi0[c];
  rx_mg_prolong_add(nx, ny, nz, e, L->phi);
  for (long c = 0; c < C->n; ++c) e[c] = C->Xs[c] - C->Xs0[c];
  rx_mg_prolong_add(nx, ny, nz, e, L->Xs);
  free(e);
  for (long c = 0; c < L->n; ++c) L->phi[c] = clampd(L->phi[c], 1e-4, 1.0);
  for (int s = 0; s < mg->nu_post; ++s) err = sweep(L, mg->omega);
  return err;
}

static int mg_ok(const rx_params *p, const rx_mg_params *mg) {
  if (!p || !mg || mg->levels < 1 || mg->levels > 16 || mg->nu_pre < 0 || mg->nu_coarse < 1 ||
      mg->max_cycles < 1 || !(mg->omega > 0.0 && mg->omega <= 1.0))
    return 0;
  if (mg->levels > 1 && mg->nu_post < 1) return 0;
  const int m = 1 << (mg->levels - 1);
  return p->nx > 0 && p->ny > 0 && p->nz > 0 && p->nx % m == 0 && p->ny % m == 0 && p->nz % m == 0;
}

static void free_levels(level *Ls, int nl) {
  for (int l = 0; l < nl; ++l) {
    level *L = &Ls[l];
    if (l > 0) {
      double *own[LEVEL_OWNED] = {L->Pf, L->phi, L->Xs, L->Pf_o, L->phi_o, L->Xs_o, L->fP, L->fphi, L->fX,
                                  L->Pf0, L->phi0, L->Xs0};
      for (int a = 0; a < LEVEL_OWNED; ++a) free(own[a]);
      free(L->R);
    }
    free(L->gP); free(L->gphi); free(L->gX); free(L->den);
  }
  free(Ls);
}

static level *alloc_levels(const rx_params *p, const rx_mg_params *mg, rx_state *s) {
  level *Ls = calloc(mg->levels, sizeof(level));
  if (!Ls) return NULL;
  int ok = 1;
  for (int l = 0; l < mg->levels; ++l) {
    level *L = &Ls[l];
    L->p = *p;
    L->p.nx = p->nx >> l;
    L->p.ny = p->ny >> l;
    L->p.nz = p->nz >> l;
    L->n = (long)L->p.nx * L->p.ny * L->p.nz;
    const size_t b = L->n * sizeof(double);
    if (l == 0) {
      L->Pf = s->Pf; L->phi = s->phi; L->Xs = s->Xs;
      L->Pf_o = s->Pf_o; L->phi_o = s->phi_o; L->Xs_o = s->Xs_o;
      L->R = s->R;
    } else {
      double **own[LEVEL_OWNED] = {&L->Pf, &L->phi, &L->Xs, &L->Pf_o, &L->phi_o, &L->Xs_o, &L->fP, &L->fphi,
                                   &L->fX, &L->Pf0, &L->phi0, &L->Xs0};
      for (int a = 0; a < LEVEL_OWNED; ++a) ok &= (*own[a] = calloc(L->n, sizeof(double))) != NULL;
      ok &= (L->R = malloc(b)) != NULL;
    }
    double **scr[LEVEL_SCRATCH] = {&L->gP, &L->gphi, &L->gX, &L->den};
    for (int a = 0; a < LEVEL_SCRATCH; ++a) ok &= (*scr[a] = malloc(b)) != NULL;
  }
  if (!ok) {
    free_levels(Ls, mg->levels);
    return NULL;
  }
  return Ls;
}

static int mg_run(const rx_params *p, const rx_mg_params *mg, rx_state *s, int ncycles, int converge, int *cycles,
                  double *change) {
  if (!mg_ok(p, mg) || ncycles < 1) return RX_EINVAL;
  level *Ls = alloc_levels(p, mg, s);
  if (!Ls) return RX_EINVAL;
  rx_begin_step(p, s);
  for (int l = 1; l < mg->levels; ++l) {
    const level *F = &Ls[l - 1];
    level *C = &Ls[l];
    rx_mg_restrict(F->p.nx, F->p.ny, F->p.nz, F->Pf_o, C->Pf_o);
    rx_mg_restrict(F->p.nx, F->p.ny, F->p.nz, F->phi_o, C->phi_o);
    rx_mg_restrict(F->p.nx, F->p.ny, F->p.nz, F->Xs_o, C->Xs_o);
  }
  int rc = RX_OK, it = 0;
  double err = 0.0;
  while (it < ncycles) {
    ++it;
    err = vcycle(Ls, 0, mg);
    if (!isfinite(err)) {
      rc = RX_ENAN;
      break;
    }
    if (converge && err < p->tol) break;
  }
  if (rc == RX_OK && converge && !(err < p->tol)) rc = RX_ENOTCONV;
  free_levels(Ls, mg->levels);
  if (cycles) *cycles = it;
  if (change) *change = err;
  return rc;
}

int rx_mg_step(const rx_params *p, const rx_mg_params *mg, rx_state *s, int *cycles, double *change) {
  return mg_run(p, mg, s, mg ? mg->max_cycles : 0, 1, cycles, change);
}

int rx_mg_cycles_n(const rx_params *p, const rx_mg_params *mg, rx_state *s, int ncycles, double *change) {
  return mg_run(p, mg, s, ncycles, 0, NULL, change);
}
