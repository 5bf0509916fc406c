/* porowave_rx.h — C ABI of the GB300 reactive porosity-wave solver (thesis Art. 3, Eqs. 8-10;
 * the pseudo-transient form of its appendix A.6 script). Fluid pressure Pf (effective pressure
 * -Pf), porosity phi and the mass fraction Xs of volatiles bound to the solid are advanced by
 * implicit physical steps of length dt, each iterated to its fixed point by one fused
 * pseudo-transient kernel per iteration:
 *   Xs_eq = clamp(beta_x Pf + Xs_max / 2, 0, Xs_max),  dXs/dt = (Xs_eq - Xs) / tau   (Eqs. 4, 10)
 *   beta_P dPf/dt = -div qD - Pf / (eta (1 - phi)) + S_r (1 - phi)(1 + dX)/(1 - Xs) dXs/dt (Eq. 8)
 *   dphi/dt = (1 - phi) (beta_phi dPf/dt + Pf / (eta (1 - phi)) - (1 + dX)/(1 - Xs) dXs/dt) (Eq. 9)
 * qD = -k0 (phi/phi0)^3 (grad Pf - rho_f g e_z) with no flux through the walls,
 * beta_P = phi beta_f + beta_d - (1 + phi) beta_s, beta_phi = beta_d - beta_s / (1 - phi),
 * S_r = 1 - rho_s / (rho_f (1 + dX)); the Pf update takes the cell's own compaction and
 * linearised reaction terms implicitly, Xs is updated local-implicitly; convergence when the
 * one-iteration change max(|dphi|, |dPf| / pf_scale, |dXs|) of an nup-th iteration is < tol.
 * All pointers are device pointers in the padded box layout of porowave_pt.h (pt_pitch_x,
 * pt_field_elems; only the cell entries are used); every call is stream-ordered on the
 * context's stream and returns after its work is done. Errors: PT_EINVAL, PT_ESPACE,
 * PT_ECUDA; rx_step returns PT_ENOTCONV at the cap and PT_ENAN for a non-finite change. */
#ifndef POROWAVE_RX_H
#define POROWAVE_RX_H

#include "porowave_pt.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rx_ctx rx_ctx;

/* Physical parameters, nondimensional (compaction length, compaction pressure, viscous time). */
typedef struct {
  double phi0;      /* background porosity of k = k0 (phi / phi0)^3          */
  double k0;        /* permeability over fluid viscosity                      */
  double eta;       /* bulk viscosity                                         */
  double rhof;      /* fluid density                                          */
  double rhos;      /* solid density                                          */
  double g;         /* gravity along -z                                       */
  double beta_d, beta_s, beta_f;  /* drained, solid, fluid compressibility    */
  double beta_x;    /* d Xs_eq / d Pf (its sign is the Clapeyron slope's)     */
  double dX;        /* solid density change with Xs (Delta X)                 */
  double xs_max;    /* largest mass fraction of volatiles in the solid        */
  double tau;       /* reaction time (1 / Damkoehler number)                  */
} rx_phys;

typedef struct {
  double dt;        /* physical time step (> 0)                                          */
  double tol;       /* convergence on the one-iteration change                           */
  double cfl_div;   /* pseudo step dtau = min(d)^2 / max(k / beta_P) / cfl_div (> 0)     */
  double pf_scale;  /* Pf's divisor in the change norm (> 0)                             */
  int32_t max_iter; /* iteration cap per physical step                                   */
  int32_t nup;      /* check (change norm, pseudo-step refresh) every nup-th iteration   */
  int32_t precision;/* PT_FP64 or PT_FP32 (iterations in single precision, as the thesis
                       ran this solver; the caller's fields stay FP64)                    */
} rx_num;

/* Caller-owned device fields (box layout): unknowns and the rate dPf/dt of the last iterate. */
typedef struct {
  double *Pf, *phi, *Xs, *R;
} rx_fields;

size_t rx_workspace_size(const pt_grid *grid, const rx_num *num);
int rx_init(rx_ctx **ctx, const pt_grid *grid, const rx_phys *phys, const rx_num *num,
            const rx_fields *fields, void *workspace, size_t bytes, void *stream);
/* One physical step to convergence (rep->iters, rep->res_v = last change norm). */
int rx_step(rx_ctx *ctx, pt_report *rep);
/* One physical step of exactly niter iterations (no convergence exit; rep as rx_step). */
int rx_iterate(rx_ctx *ctx, int32_t niter, pt_report *rep);
/* ---- Geometric multigrid acceleration (the thesis's future-work section: PT iterations with
 * local pseudo steps are weighted Jacobi iterations, which geometric multigrid accelerates; the
 * nonlinearity by the full approximation scheme, FAS). The smoother is the iteration above with
 * the local pseudo step dtau = omega beta_P / Dk (Dk = Jacobi diagonal of the Darcy operator,
 * the cell's own terms implicit); coarse grids are 2 x 2 x 2 agglomerations (nx, ny, nz
 * divisible by 2^(levels-1)), restriction = mean of the 8 children (iterate and residual),
 * prolongation = trilinear interpolation of the coarse correction (neighbour held at the wall).
 * A V-cycle on level l: nu_pre sweeps, restriction, FAS source f_c = mean(r) - g_c(u0_c), the
 * cycle on l + 1 (nu_coarse sweeps on the coarsest), correction, nu_post sweeps. The change of a
 * cycle is max(|dphi|, |dPf| / pf_scale, |dXs|) of its last sweep on the finest grid; R is that
 * sweep's rate. The converged step is the fixed point of the plain iteration. */
typedef struct {
  int32_t levels;     /* grids in the hierarchy, 1..16 (1 = the smoother alone)              */
  int32_t nu_pre;     /* sweeps before the coarse-grid correction (>= 0)                     */
  int32_t nu_post;    /* sweeps after it (>= 1 when levels > 1)                              */
  int32_t nu_coarse;  /* sweeps on the coarsest grid (>= 1)                                  */
  int32_t max_cycles; /* V-cycle cap of rx_mg_step (>= 1)                                    */
  double omega;       /* Jacobi weight of the Darcy part, 0 < omega <= 1 (6/7: 3-D optimum)  */
} rx_mg;

/* Workspace of a multigrid context: rx_workspace_size plus 15 arrays per coarse level; 0 for an
 * invalid grid, numerics or hierarchy (a dimension not divisible by 2^(levels-1)). */
size_t rx_mg_workspace_size(const pt_grid *grid, const rx_num *num, const rx_mg *mg);
/* As rx_init, with the hierarchy; the context also runs rx_step / rx_iterate (plain PT). */
int rx_mg_init(rx_ctx **ctx, const pt_grid *grid, const rx_phys *phys, const rx_num *num,
               const rx_mg *mg, const rx_fields *fields, void *workspace, size_t bytes, void *stream);
/* One physical step by V-cycles until the change is < num.tol (rep->iters = cycles; PT_ENOTCONV
 * at max_cycles, PT_ENAN for a non-finite change, PT_EINVAL on a plain context). */
int rx_mg_step(rx_ctx *ctx, pt_report *rep);
/* One physical step of exactly ncycles V-cycles (rep as rx_mg_step). */
int rx_mg_cycles(rx_ctx *ctx, int32_t ncycles, pt_report *rep);

/* Launches of the library's kernels so far (benchmark accounting). */
long long rx_launch_count(const rx_ctx *ctx);
void rx_destroy(rx_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
