/* rx_oracle.h — plain FP64 CPU oracle of the reactive porosity-wave solver (thesis Art. 3,
 * Eqs. 8-10, appendix A.6). TEST INFRASTRUCTURE ONLY; see rx_oracle.c for the method. */
#ifndef RX_ORACLE_H
#define RX_ORACLE_H

enum { RX_OK = 0, RX_EINVAL = -1, RX_ENOTCONV = -2, RX_ENAN = -3 };

typedef struct {
  int nx, ny, nz;
  double lx, ly, lz;
  /* physics (nondimensional: compaction length, compaction pressure, viscous time) */
  double phi0;      /* background porosity (k = k0 (phi / phi0)^3)                       */
  double k0;        /* permeability over fluid viscosity                                 */
  double eta;       /* bulk viscosity                                                    */
  double rhof, rhos;  /* fluid and solid density                                        */
  double g;           /* gravity (along -z)                                              */
  double beta_d, beta_s, beta_f;  /* drained, solid and fluid compressibilities          */
  double beta_x;    /* d Xs_eq / d Pf (sign: Clapeyron slope)                            */
  double dX;        /* solid density change with Xs (Delta X)                            */
  double xs_max;    /* largest mass fraction of volatiles in the solid                   */
  double tau;       /* reaction time (1 / Da in viscous time units)                      */
  /* numerics */
  double dt, tol, cfl_div, pf_scale;
  int max_iter, nup;
} rx_params;

typedef struct {
  double *Pf, *phi, *Xs, *R;      /* iterate; R = dPf/dt at the last iterate (output)  */
  double *Pf_o, *phi_o, *Xs_o;    /* old step                                           */
  double dtau;                    /* current pseudo step of Pf                          */
} rx_state;

double rx_perm(const rx_params *p, double phi);
double rx_beta_p(const rx_params *p, double phi);
double rx_xseq(const rx_params *p, double Pf);
void rx_div_qd(const rx_params *p, const double *Pf, const double *phi, double *divq);
double rx_pseudo_step(const rx_params *p, const double *phi);
/* old-step copies and the first pseudo step */
int rx_begin_step(const rx_params *p, rx_state *s);
/* PT iteration number `it` (1-based); *change = the one-iteration change norm */
int rx_iteration(const rx_params *p, rx_state *s, int it, double *change);
/* one physical step: begin, iterate until the change norm of an nup-th iteration is < tol */
int rx_step(const rx_params *p, rx_state *s, int *iters, double *change);
/* begin a step and run exactly niter iterations */
int rx_iterate_n(const rx_params *p, rx_state *s, int niter, double *change);

#endif
