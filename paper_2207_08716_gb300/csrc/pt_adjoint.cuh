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
  // power-law rheology (Eq. 24): mu varies, the Picard row F_mu = log mu - log mu*(tau_II) joins
  int powerlaw;
  double Gdt;                           // G dtS of the step (xi = mu / Gdt)
  double rtau0_2, pw;                   // 1 / tau0^2, (n - 1) / 2
  double r_eta0, dtauv_fac, dtaupt_fac; // 1 / eta0, dtau_V = fac / mu, dtau_Pt = fac * mu
};

struct AdjState {                       // converged state of the step (frozen during its solve)
  const double *Vx, *Vy, *Vz, *Pt, *Pf, *phi;
  const double *mu;                     // Picard state (power law; null otherwise)
};

// Power-law coefficients of one step (its converged state), see pt_adjoint_kernels.cu.
struct AdjPrepPL {
  double *mc, *cc, *cplL, *imu;         // 2 mu/(1+xi), 1/(eta(1-phi)), beta_phi + dt/eta, 1/mu
  double *Qxx, *Qyy, *Qzz;              // dm/dmu times the state's deviatoric strain rates
  double *sTxx, *sTyy, *sTzz;           // m f tau_ii: centre part of the pseudo-stress per lambda_mu
  double *Axy, *Axz, *Ayz;              // f a_e / 2 per centre (a_e: edge stresses averaged to it)
  double *me_xy, *me_xz, *me_yz;        // edge moduli
  double *P_xy, *P_xz, *P_yz;           // (dm/dmu)_e eps_e / 4 on edges
  double *iDmu, *cmu, *cmuL;            // 1 / diagonal of row mu; (Pt-Pf) cc / mu; (Pt-Pf) dt phi / (eta0 mu^2)
  double *dtvx, *dtvy, *dtvz;           // velocity pseudo-steps at faces (mean of the two centres')
  double *fTQ;                          // f sum_ii tau_ii Q_ii (own part of row mu's lambda_mu term)
};
// Edges of one adjoint iteration (power law): pseudo-stress sigma_e from lambda_mu, the edge's
// adjoint stress m_e (eps_e(lambda_V) - sigma_e / 2) and Z_e = sigma_e - 2 eps_e(lambda_V).
struct AdjEdgeIn {
  const double *Lx, *Ly, *Lz, *lM, *Axy, *Axz, *Ayz, *me_xy, *me_xz, *me_yz;
};
struct AdjEdgeOut {
  double *txy, *txz, *tyz, *Zxy, *Zxz, *Zyz;
};
struct AdjMuIn {                        // row mu inputs of the cells kernel (power law)
  const double *lM, *gM, *Zxy, *Zxz, *Zyz;
  double *lM1;                          // next lambda_mu
  double *rM;                           // residual of row mu (written when non-null)
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
  const double *dtvx, *dtvy, *dtvz;     // per-face pseudo-steps (power law), else null: uniform
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

// ---- power law
// two passes (edges, then centres); tau_e are three scratch edge arrays for the state's edge stresses
void adj_prep_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const double* K0,
                 const AdjPrep& out, const AdjPrepPL& pl, double* tau_xy, double* tau_xz, double* tau_yz);
void adj_edges_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjEdgeIn& in,
                  const AdjEdgeOut& out);
void adj_cells_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
                  const AdjCellOut& out, const AdjPrepPL& pl, const AdjMuIn& mu, unsigned long long* red,
                  int check);
// sum over the grid of d(lambda . F)/d(G dtS) into *acc (one double, atomically), for the carry of
// the dtS = max(mu_prev) / (G xsi_w) dependence
void adj_dgdt_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u,
                 const AdjPrepPL& pl, const double* Lx, const double* Ly, const double* Lz, const double* lM,
                 const double* Zxy, const double* Zxz, const double* Zyz, double* acc);
// red[RED_MUMAX] = max(mu) over the cells (bit pattern), then red[RED_ARG] = the smallest box
// index of a cell holding it
void adj_argmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* mu, unsigned long long* red);
// gM[red[RED_ARG]] += scale * (*acc) (one thread; nothing when no index was found)
void adj_add_at(cudaStream_t s, Box b, double* gM, const unsigned long long* red, const double* acc,
                double scale);
constexpr int RED_ARG = 6;   // reduction slot of the argmax index (adjoint carry)

}  // namespace pt
