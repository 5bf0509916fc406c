/* rx_mg_oracle.h — plain FP64 CPU oracle of the geometric-multigrid (FAS) acceleration of the
 * reactive porosity-wave step (thesis Art. 3, Eqs. 8-10; the thesis's future-work section on
 * multigrid-accelerated pseudo-transient iterations). TEST INFRASTRUCTURE ONLY; see
 * rx_mg_oracle.c for the method. */
#ifndef RX_MG_ORACLE_H
#define RX_MG_ORACLE_H

#include "rx_oracle.h"

typedef struct {
  int levels;       /* grids in the hierarchy (1 = the smoother alone)                       */
  int nu_pre;       /* smoothing sweeps before the coarse-grid correction                    */
  int nu_post;      /* smoothing sweeps after it (>= 1 when levels > 1)                      */
  int nu_coarse;    /* sweeps on the coarsest grid (>= 1)                                    */
  int max_cycles;   /* V-cycle cap per physical step                                         */
  double omega;     /* Jacobi weight of the diffusion part of the pseudo step (0 < omega <= 1) */
} rx_mg_params;

/* Transfer operators on one level pair (fine nx x ny x nz, coarse nx/2 x ny/2 x nz/2). */
void rx_mg_restrict(int nx, int ny, int nz, const double *fine, double *coarse);
void rx_mg_prolong_add(int nx, int ny, int nz, const double *coarse_e, double *fine);
/* The three step equations as "target - current" on a grid with FAS sources f (nullable):
 * gP (rate units), gphi, gX, and the Jacobi denominator den of gP; R = the rate. */
void rx_mg_equations(const rx_params *p, const double *Pf, const double *phi, const double *Xs,
                     const double *Pf_o, const double *phi_o, const double *Xs_o, const double *fP,
                     const double *fphi, const double *fX, double omega, double *gP, double *gphi,
                     double *gX, double *den, double *R);
/* one physical step: begin, V-cycles until the change of the last finest-grid sweep is < tol */
int rx_mg_step(const rx_params *p, const rx_mg_params *mg, rx_state *s, int *cycles, double *change);
/* begin a step and run exactly ncycles V-cycles */
int rx_mg_cycles_n(const rx_params *p, const rx_mg_params *mg, rx_state *s, int ncycles, double *change);

#endif
