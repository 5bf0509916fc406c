/* pt_oracle.h — interface of the plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY. The oracle is the slow, obviously-correct reference that the CUDA
 * path is checked against. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * may load it. It shares no code, header or constant with the CUDA library.
 *
 * Model: thesis Art. 1, Section 2.1 (Eqs. 1-11) in the pseudo-transient form of Section 2.2
 * (Eqs. 17-27), discretised on the staggered grid of Fig. 1 as in the appendix's 3-D
 * two-phase input script, with the readings listed in the design notes.
 *
 * Storage: every field is its own array in its natural staggered size, x fastest:
 *   centres          nx     * ny     * nz        (Pt, Pf, phi, mu, eta, txx, tyy, tzz, ...)
 *   x-faces          (nx+1) * ny     * nz        (Vx, Rx)
 *   y-faces          nx     * (ny+1) * nz        (Vy, Ry)
 *   z-faces          nx     * ny     * (nz+1)    (Vz, Rz)
 *   xy-edges         (nx+1) * (ny+1) * nz        (txy)
 *   xz-edges         (nx+1) * ny     * (nz+1)    (txz)
 *   yz-edges         nx     * (ny+1) * (nz+1)    (tyz)
 */
#ifndef PT_ORACLE_H
#define PT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOTCONV = -2, OR_ENAN = -3 };

typedef struct {
  /* grid: cell-centred, dx = lx / nx */
  int nx, ny, nz;
  double lx, ly, lz;
  /* physics (Table 2 symbols) */
  double phi0, k0, mu0, eta0, R_weak, n_pow, tau0, alpha, B, beta_d, beta_phi, G, rhof_g, rhos_g;
  int powerlaw_on, compaction_on;
  /* numerics */
  double dt, tol;
  int max_iter, nup;
  double damp_x, damp_y, damp_z, rho_i, beta_n, rel_mu, rel_eta, cfl_v, cfl_pf, dtpt_scale;
  double xsi_w;       /* wanted largest xi = mu / (G dtS) of the stress sub-step */
  /* oracle-only switch: 0 freezes the solid (no momentum, V stays as given). Used by the
   * linear-diffusion-limit pin, where the P-Pf system decouples from the mechanics. */
  int mech_on;
  /* applied horizontal background shear stress (Eqs. 32-33; 0 = none): the background flow
   * V_bg = (tau_bg / mu0) (y - ly/2) e_x adds tau_bg / (2 mu0) to the xy strain rate at every
   * xy-edge, the wall edges included, where the unknown velocity's part is zero (free slip) */
  double tau_bg;
} or_params;

typedef struct {
  double *Vx, *Vy, *Vz;                        /* solid velocity (faces)                 */
  double *Pt, *Pf, *phi;                       /* total, fluid pressure, porosity        */
  double *txx, *tyy, *tzz, *txy, *txz, *tyz;   /* deviatoric stress at end of step       */
  double *mu, *eta;                            /* Picard shear and bulk viscosity        */
  double *Rx, *Ry, *Rz;                        /* damped momentum residuals (faces)      */
  double *Pto, *Pfo, *Lo;                      /* old step: Pt, Pf, log(1 - phi)         */
  double *txxo, *tyyo, *tzzo, *txyo, *txzo, *tyzo;  /* old-step stresses                 */
  const double *logk;                          /* known log-permeability field or NULL   */
  /* stress sub-stepping (appendix two-phase script): dtS = max(mu) / (G xsi_w); the old
   * stresses are refreshed when the accumulated time dt_cum reaches dtS or at the first step */
  double dtS, dt_cum;
  int nsteps;                                  /* physical steps begun so far            */
} or_state;

/* residual norms (max-norms), Section "c4.10" of the design notes */
typedef struct { double r_v, r_pt, r_pf, r_pic; } or_res;

/* Initial Picard state from porosity: mu = mu0, eta = eta0 * mu / phi (Eq. 26, R = 1). */
int or_init_viscosities(const or_params *p, or_state *s);
/* Old-state snapshot at the start of a physical step: Pto, Pfo, Lo; dtS from max(mu); the old
 * stresses are refreshed at the first step and whenever dt_cum >= dtS (dt_cum is then reset). */
int or_begin_step(const or_params *p, or_state *s);
/* One PT iteration number `it` (1-based within the step). Picard update and residual norms
 * are taken when it % nup == 0 (`res` is then filled and *checked = 1). */
int or_iteration(const or_params *p, or_state *s, int it, or_res *res, int *checked);
/* Stresses of the final state of the step, written to s->txx ... s->tyz; dt_cum += dt. */
int or_end_step(const or_params *p, or_state *s);
/* One physical step: begin, iterate to tol or max_iter, end. Returns OR_ENOTCONV at the cap. */
int or_step(const or_params *p, or_state *s, int *iters, or_res *res);
/* Iterate `niter` PT iterations from iteration number it0+1 (no convergence exit). */
int or_iterate_n(const or_params *p, or_state *s, int it0, int niter, or_res *res);

/* ---- building blocks (exposed for the unit pins) ---- */
void or_coefficients(const or_params *p, const double *phi, const double *logk,
                     double *perm, double *rog);
void or_darcy(const or_params *p, const double *Pf, const double *perm,
              double *qx, double *qy, double *qz, double *divqD);
void or_divergence(const or_params *p, const double *Vx, const double *Vy, const double *Vz,
                   const double *Pt, const double *Pf, const double *Pto, const double *Pfo,
                   const double *phi, const double *eta, double *divV, double *divVn);
void or_stress(const or_params *p, double dtS, const double *Vx, const double *Vy, const double *Vz,
               const double *divV, const double *divVn, const double *mu,
               const double *txxo, const double *tyyo, const double *tzzo,
               const double *txyo, const double *txzo, const double *tyzo,
               double *txx, double *tyy, double *tzz, double *txy, double *txz, double *tyz);
void or_momentum(const or_params *p, const double *txx, const double *tyy, const double *tzz,
                 const double *txy, const double *txz, const double *tyz,
                 const double *Pt, const double *rog, double *Fx, double *Fy, double *Fz);
void or_advection(const or_params *p, const double *Vx, const double *Vy, const double *Vz,
                  const double *phi, double *adv);
void or_tau_II(const or_params *p, const double *txx, const double *tyy, const double *tzz,
               const double *txy, const double *txz, const double *tyz, double *tII);
/* Residual of the implicit step at the current state (for the brute-force Newton pin):
 * out_V* = momentum F on every face (0 on boundary faces), out_pt = divVn, out_pf = fluid
 * pressure residual, out_L = log(1-phi) - [porosity update target], out_mu = log mu - log mu*,
 * out_eta = log eta - log eta*. */
int or_system_residual(const or_params *p, const or_state *s,
                       double *out_Vx, double *out_Vy, double *out_Vz, double *out_pt,
                       double *out_pf, double *out_L, double *out_mu, double *out_eta);

/* OpenMP threads the oracle's loops use. */
int or_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
