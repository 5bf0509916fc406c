// pt_adjoint.cuh — argument structs and launchers of the adjoint kernels (pt_adjoint_kernels.cu).
#pragma once

#include "pt_common.cuh"

namespace pt {

struct AdjCoef {
  double rdx, rdy, rdz;
  double m2;                    // 2 mu0 / (1 + xi): uniform shear coefficient (mu = mu0)
  double r_eta0mu0;             // 1 / (eta0 mu0)
  double bd_rdt, bd_rdt_a, bda_B_rdt, beta_phi, dt;
  double idtp;                  // 1 / dtau_Pt at mu0
  double ifac_pf;               // 1 / dtau_Pf = kmax * ifac_pf
  double rphi0, k0;
  double buoy;                  // (rho_f - rho_BG) g
  double drho_g;                // (rho_f - rho_s) g
  double rrho_i, damp_x, damp_y, damp_z, dtauv;
};
struct AdjState {               // converged state of the step (frozen)
  const double *Vx, *Vy, *Vz, *Pt, *Pf, *phi;
};
struct AdjCellIn {
  const double *Lx, *Ly, *Lz, *lP, *lF, *lL, *gP, *gF, *gphi, *K0;
};
struct AdjCellOut {
  double *txx, *tyy, *tzz, *txy, *txz, *tyz, *lP, *lF, *lL, *gtheta;
};
struct AdjFaceIn {
  const double *txx, *tyy, *tzz, *txy, *txz, *tyz, *lP1, *lL;
};
struct AdjCarry {
  const double *lP, *lF, *lL, *gtheta, *phi_o;
  double *grad, *gP, *gF, *gphi;
};

void adj_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
               const AdjCellOut& out, unsigned long long* red, int check);
void adj_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjFaceIn& in,
               double* Lx, double* Ly, double* Lz, double* Rx, double* Ry, double* Rz, unsigned long long* red,
               int check);
void adj_carry(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjCarry& a);
// red[RED_GMAX] = max(red[RED_GMAX], max |gP|, |gF|, |gphi| over the cells)
void adj_gmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* gP, const double* gF, const double* gphi,
              unsigned long long* red);

}  // namespace pt
