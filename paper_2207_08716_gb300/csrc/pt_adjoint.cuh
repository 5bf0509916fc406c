// pt_adjoint.cuh — argument structs and host launchers of the adjoint kernels
// (pt_adjoint_kernels.cu): the transposed system J_F(u)^T lambda = g of one converged implicit
// step, solved by pseudo-transient iteration.
#pragma once

#include "pt_common.cuh"

namespace pt {

// Per-run scalars (FP64). In the adjoint's scope mu = mu0 everywhere, so the viscoelastic
// modulus, the velocity pseudo-step and the total-pressure pseudo-step are uniform.
struct AdjCoef {
  double rdx, rdy, rdz;
  double m2, third;                     // 2 mu0 / (1 + xi), 1/3
  double hm2rdx, hm2rdy, hm2rdz;        // m2 / 2 / d_i (edge stresses)
  double r_eta0mu0;                     // 1 / (eta0 mu0)
  double bd_rdt, bd_rdt_a, bda_B_rdt, beta_phi, dt, dt_r;   // dt_r = dt / (eta0 mu0)
  double idtp;                          // 1 / dtau_Pt
  double ifac_pf;                       // dtau_Pf = 1 / (kmax ifac_pf)
  double rphi0, k0;
  double buoy;                          // (rho_f - rho_BG) g
  double hdrho_g;                       // (rho_f - rho_s) g / 2
  double hdt_rdx, hdt_rdy, hdt_rdz;     // dt / 2 / d_i (advection)
  double rrho_i, damp_x, damp_y, damp_z, dtauv;
};

struct AdjState {                       // converged state of the step (frozen during its solve)
  const double *Vx, *Vy, *Vz, *Pt, *Pf, *phi;
};

// Coefficients of one step's transposed system, from its converged state (one launch per step).
struct AdjPrep {
  double *W;                            // 1 / (1 - phi)
  double *cP, *cF;                      // inverse local-implicit diagonals of rows Pt, Pf
  double *Dg, *iD;                      // diagonal of row phi and its inverse
  double *aPF;                          // (Pt - Pf) d(1/(eta(1-phi)))/dphi
  double *a3k;                          // 3 k / phi  (dk/dphi)
  double *kfx, *kfy, *kfz;              // Darcy face coefficients (k_l + k_r) / 2 / d^2 (0 on walls)
  double *gkx, *gky, *gkz;              // -(dPf/dn + buoyancy) / 2 / d on faces (d q / d k)
  double *bfx, *bfy, *bfz;              // -dt (phi_r - phi_l) / 2 / d on faces (advection)
  const double *lL;                     // warm-start lambda_L ...
  double *mL;                           // ... and lambda_L / (1 - phi) for it
};

struct AdjCellIn {
  const double *Lx, *Ly, *Lz, *lP, *lF, *lL, *mL, *gP, *gF, *gphi, *K0;
  const double *W, *cP, *cF, *Dg, *iD, *aPF, *a3k, *kfx, *kfy, *kfz, *gkx, *gky, *gkz;
};
struct AdjCellOut {
  double *txx, *tyy, *tzz, *txy, *txz, *tyz, *lP, *lF, *lL, *mL;
  double *gtheta;                       // k (dF_Pf/dk)^T lambda_F (written when non-null)
  double *rP, *rF, *rL;                 // residual rows (J^T lambda - g), written when non-null
};
struct AdjFaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *lP1, *mL, *bfx, *bfy, *bfz;
  double *rx, *ry, *rz;                 // residual rows of lambda_V, written when non-null
  int update;                           // 0: evaluate only (no R / lambda_V update)
};
struct AdjCarry {
  const double *lP, *lF, *lL, *gtheta, *phi_o;
  double *grad, *gP, *gF, *gphi;
};

void adj_prep(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const double* K0,
              const AdjPrep& out);
void adj_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
               const AdjCellOut& out, unsigned long long* red, int check);
void adj_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjFaceIn& in, double* Lx,
               double* Ly, double* Lz, double* Rx, double* Ry, double* Rz, unsigned long long* red, int check);
void adj_carry(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjCarry& a);
// red[RED_GMAX] = max(red[RED_GMAX], max |gP|, |gF|, |gphi| over the cells)
void adj_gmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* gP, const double* gF, const double* gphi,
              unsigned long long* red);

}  // namespace pt
