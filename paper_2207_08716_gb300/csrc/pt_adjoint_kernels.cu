// pt_adjoint_kernels.cu — discrete adjoint of the converged implicit step (Art. 1, Eqs. 17-26;
// the thesis has no adjoint: the gradient of a final-porosity misfit w.r.t. the log-k field).
//
// Each physical step solves F(u; u_o, theta) = 0 for u = (V, Pt, Pf, phi) (Eqs. 17-22 with the
// power law off, no weakening switch, beta_n = 0 and fixed old stresses, so eta = eta0 mu0 / phi).
// For an objective J(phi^N) the adjoint of step n solves J_F(u^n)^T lambda = g^n with the same
// pseudo-transient scheme as the forward solve, on the transposed staggered stencils:
//   row V  (faces):  A lambda_V - grad lambda_P + (d adv / d V)^T lambda_L
//                    (A: the symmetric viscoelastic operator; damped PT, as the forward V)
//   row Pt (centres): div lambda_V + (beta_d/dt + c) lambda_P - (beta_d alpha/dt + c) lambda_F
//                    - (beta_phi + dt/eta) lambda_L - g_P     (local-implicit PT)
//   row Pf (centres): K lambda_F + (beta_d alpha/(B dt) + c) lambda_F - (beta_d alpha/dt + c) lambda_P
//                    + (beta_phi + dt/eta) lambda_L - g_F      (K: the symmetric Darcy operator)
//   row phi(centres): buoyancy, compaction, dk/dphi and advection transposes; lambda_L from its
//                    own diagonal dF_L/dphi = -1/(1-phi) + ... (Jacobi)
// with c = phi / ((1-phi) eta0 mu0) and k = k0 e^theta (phi/phi0)^3.
//
// GB300 form: FP64 throughput (not HBM) bounds these stencils, so everything that depends only
// on the frozen converged state — 1/(1-phi), k and its face averages, dPf/dn, the row diagonals
// and their inverses — is computed once per step by k_adj_prep, and the iteration kernels are
// left with multiply-adds: no division and no k(phi) evaluation per iteration.
#include "pt_adjoint.cuh"

namespace pt {

namespace {
__device__ inline double pos_max_d(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(ia > ib ? ia : ib);
}
__device__ inline double kperm(const AdjCoef& c, const double* K0, long long q, double ph) {
  const double r = ph * c.rphi0;
  return (K0 ? K0[q] : c.k0) * r * r * r;
}
}  // namespace

// Per-step coefficients from the converged state u (cells i < nx ... and their lower faces).
__global__ void __launch_bounds__(256) k_adj_prep(Box b, AdjCoef c, AdjState u, const double* __restrict__ K0,
                                                  AdjPrep o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  // lower faces of the cell (i, j, k): interior faces only, zero elsewhere
  {
    double kf = 0.0, gk = 0.0, bf = 0.0;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {
      const double pl = u.phi[q - 1], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - 1, pl) + kperm(c, K0, q, pr)) * c.rdx * c.rdx;
      gk = -0.5 * (u.Pf[q] - u.Pf[q - 1]) * c.rdx * c.rdx;
      bf = -c.hdt_rdx * (pr - pl);
    }
    o.kfx[q] = kf; o.gkx[q] = gk; o.bfx[q] = bf;
  }
  {
    double kf = 0.0, gk = 0.0, bf = 0.0;
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {
      const double pl = u.phi[q - px], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - px, pl) + kperm(c, K0, q, pr)) * c.rdy * c.rdy;
      gk = -0.5 * (u.Pf[q] - u.Pf[q - px]) * c.rdy * c.rdy;
      bf = -c.hdt_rdy * (pr - pl);
    }
    o.kfy[q] = kf; o.gky[q] = gk; o.bfy[q] = bf;
  }
  {
    double kf = 0.0, gk = 0.0, bf = 0.0;
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {
      const double pl = u.phi[q - pxy], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - pxy, pl) + kperm(c, K0, q, pr)) * c.rdz * c.rdz;
      gk = -0.5 * ((u.Pf[q] - u.Pf[q - pxy]) * c.rdz + c.buoy) * c.rdz;
      bf = -c.hdt_rdz * (pr - pl);
    }
    o.kfz[q] = kf; o.gkz[q] = gk; o.bfz[q] = bf;
  }
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const double ph = u.phi[q];
  const double w = 1.0 / (1.0 - ph);
  const double cc = ph * w * c.r_eta0mu0;
  const double kc = kperm(c, K0, q, ph);
  double kmax = kc;
  if (i > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - 1, u.phi[q - 1]));
  if (i < b.nx - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + 1, u.phi[q + 1]));
  if (j > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - px, u.phi[q - px]));
  if (j < b.ny - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + px, u.phi[q + px]));
  if (k > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - pxy, u.phi[q - pxy]));
  if (k < b.nz - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + pxy, u.phi[q + pxy]));
  const double Pt = u.Pt[q], Pf = u.Pf[q];
  o.W[q] = w;
  o.cP[q] = 1.0 / (c.idtp + c.bd_rdt + cc);
  o.cF[q] = 1.0 / (kmax * c.ifac_pf + c.bda_B_rdt + cc);
  o.aPF[q] = (Pt - Pf) * w * w * c.r_eta0mu0;
  o.a3k[q] = 3.0 * kc / ph;
  // diagonal of row phi: d/dphi [log(1-phi) + dt (Pf-Pt) phi/(eta0 mu0) + dt S / (2 (1-phi))],
  // S = sum over the cell's interior faces of V (om_r - om_l) / d, om = 1 - phi
  const double omc = 1.0 - ph;
  double S = 0.0, dS = 0.0;
  if (i > 0) { S += u.Vx[q] * (omc - (1.0 - u.phi[q - 1])) * c.rdx; dS -= u.Vx[q] * c.rdx; }
  if (i < b.nx - 1) { S += u.Vx[q + 1] * ((1.0 - u.phi[q + 1]) - omc) * c.rdx; dS += u.Vx[q + 1] * c.rdx; }
  if (j > 0) { S += u.Vy[q] * (omc - (1.0 - u.phi[q - px])) * c.rdy; dS -= u.Vy[q] * c.rdy; }
  if (j < b.ny - 1) { S += u.Vy[q + px] * ((1.0 - u.phi[q + px]) - omc) * c.rdy; dS += u.Vy[q + px] * c.rdy; }
  if (k > 0) { S += u.Vz[q] * (omc - (1.0 - u.phi[q - pxy])) * c.rdz; dS -= u.Vz[q] * c.rdz; }
  if (k < b.nz - 1) { S += u.Vz[q + pxy] * ((1.0 - u.phi[q + pxy]) - omc) * c.rdz; dS += u.Vz[q + pxy] * c.rdz; }
  const double diag = -w + c.dt_r * (Pf - Pt) + c.dt * 0.5 * (w * w * S + w * dS);
  o.Dg[q] = diag;
  o.iD[q] = 1.0 / diag;
  o.mL[q] = o.lL[q] * w;
}

// Cells: adjoint stresses of lambda_V at centres and the cell's lower edges, and the centre
// updates of lambda_P, lambda_F, lambda_L.
__global__ void __launch_bounds__(256) k_adj_cells(Box b, AdjCoef c, AdjState u, AdjCellIn in, AdjCellOut out,
                                                   unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0, r_l = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (k < b.nz) {
      double t = 0.0;
      if (i > 0 && i < b.nx && j > 0 && j < b.ny)
        t = c.hm2rdy * (in.Lx[q] - in.Lx[q - px]) + c.hm2rdx * (in.Ly[q] - in.Ly[q - 1]);
      out.txy[q] = t;
    }
    if (j < b.ny) {
      double t = 0.0;
      if (i > 0 && i < b.nx && k > 0 && k < b.nz)
        t = c.hm2rdz * (in.Lx[q] - in.Lx[q - pxy]) + c.hm2rdx * (in.Lz[q] - in.Lz[q - 1]);
      out.txz[q] = t;
    }
    if (i < b.nx) {
      double t = 0.0;
      if (j > 0 && j < b.ny && k > 0 && k < b.nz)
        t = c.hm2rdz * (in.Ly[q] - in.Ly[q - pxy]) + c.hm2rdy * (in.Lz[q] - in.Lz[q - px]);
      out.tyz[q] = t;
    }
    if (i < b.nx && j < b.ny && k < b.nz) {
      const double ph = u.phi[q];
      const double cc = ph * in.W[q] * c.r_eta0mu0;
      const double lP = in.lP[q], lF = in.lF[q], lL = in.lL[q];
      // lambda_V at the cell's faces (wall faces are not unknowns and stay zero)
      const double Lz0 = in.Lz[q], Lz1 = in.Lz[q + pxy];
      const double gx = (in.Lx[q + 1] - in.Lx[q]) * c.rdx, gy = (in.Ly[q + px] - in.Ly[q]) * c.rdy;
      const double gz = (Lz1 - Lz0) * c.rdz;
      const double divL = gx + gy + gz;
      const double d3 = divL * c.third;
      out.txx[q] = c.m2 * (gx - d3);
      out.tyy[q] = c.m2 * (gy - d3);
      out.tzz[q] = c.m2 * (gz - d3);
      // ---- row Pt
      const double cplP = c.bd_rdt_a + cc, cplL = c.beta_phi + c.dt_r * ph;
      const double resP = divL + (c.bd_rdt + cc) * lP - cplP * lF - cplL * lL - in.gP[q];
      out.lP[q] = lP - in.cP[q] * resP;
      // ---- row Pf: K lambda_F and (dq/dk)^T lambda_F over the six faces; the advection
      // transpose of row phi over the same faces
      double Klf = 0.0, dkT = 0.0, offx = 0.0, offy = 0.0, offz = 0.0;
      if (i > 0) {
        const double dn = in.lF[q - 1] - lF;
        Klf -= in.kfx[q] * dn;
        dkT += in.gkx[q] * dn;
        offx -= u.Vx[q] * in.mL[q - 1];
      }
      if (i < b.nx - 1) {
        const double dn = in.lF[q + 1] - lF;
        Klf -= in.kfx[q + 1] * dn;
        dkT -= in.gkx[q + 1] * dn;
        offx += u.Vx[q + 1] * in.mL[q + 1];
      }
      if (j > 0) {
        const double dn = in.lF[q - px] - lF;
        Klf -= in.kfy[q] * dn;
        dkT += in.gky[q] * dn;
        offy -= u.Vy[q] * in.mL[q - px];
      }
      if (j < b.ny - 1) {
        const double dn = in.lF[q + px] - lF;
        Klf -= in.kfy[q + px] * dn;
        dkT -= in.gky[q + px] * dn;
        offy += u.Vy[q + px] * in.mL[q + px];
      }
      if (k > 0) {
        const double dn = in.lF[q - pxy] - lF;
        Klf -= in.kfz[q] * dn;
        dkT += in.gkz[q] * dn;
        offz -= u.Vz[q] * in.mL[q - pxy];
      }
      if (k < b.nz - 1) {
        const double dn = in.lF[q + pxy] - lF;
        Klf -= in.kfz[q + pxy] * dn;
        dkT -= in.gkz[q + pxy] * dn;
        offz += u.Vz[q + pxy] * in.mL[q + pxy];
      }
      const double off = offx * c.hdt_rdx + offy * c.hdt_rdy + offz * c.hdt_rdz;
      const double resF = Klf + (c.bda_B_rdt + cc) * lF - cplP * lP + cplL * lL - in.gF[q];
      out.lF[q] = lF - in.cF[q] * resF;
      const double a3k = in.a3k[q];
      if (out.gtheta) out.gtheta[q] = a3k * ph * c.third * dkT;   // k (dq/dk)^T lambda_F
      // ---- row phi: buoyancy (Eq. 19), compaction (Eqs. 17-18), k(phi) (Eq. 23), advection
      const double sL = -c.hdrho_g * (Lz0 + Lz1) + in.aPF[q] * (lP - lF) + a3k * dkT + off - in.gphi[q];
      const double lLn = -in.iD[q] * sL;
      out.lL[q] = lLn;
      out.mL[q] = lLn * in.W[q];
      if (check || out.rL) {
        const double resL = sL + in.Dg[q] * lL;
        if (out.rL) {
          out.rP[q] = resP;
          out.rF[q] = resF;
          out.rL[q] = resL;
        }
        r_pt = fabs(resP);
        r_pf = fabs(resF);
        r_l = fabs(resL);
      }
    }
  }
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
    block_max_atomic(r_l, red + RED_PIC);
  }
}

// Faces: row V with lambda_P1 and mL = lambda_L / (1 - phi); damped R, lambda_V update.
__global__ void __launch_bounds__(256) k_adj_faces(Box b, AdjCoef c, AdjFaceIn in, double* Lx, double* Ly,
                                                   double* Lz, double* Rx, double* Ry, double* Rz,
                                                   unsigned long long* red, int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const bool fx = i > 0 && i < b.nx && j < b.ny && k < b.nz;
    const bool fy = j > 0 && j < b.ny && i < b.nx && k < b.nz;
    const bool fz = k > 0 && k < b.nz && i < b.nx && j < b.ny;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, Rx1 = 0.0, Ry1 = 0.0, Rz1 = 0.0, Lx1 = 0.0, Ly1 = 0.0, Lz1 = 0.0;
    if (fx) {
      Fx = (in.txx[q] - in.txx[q - 1]) * c.rdx + (in.txy[q + px] - in.txy[q]) * c.rdy +
           (in.txz[q + pxy] - in.txz[q]) * c.rdz - (in.lP1[q] - in.lP1[q - 1]) * c.rdx +
           in.bfx[q] * (in.mL[q - 1] + in.mL[q]);
      if (in.update) {
        Rx1 = Fx * c.rrho_i + c.damp_x * Rx[q];
        Lx1 = Lx[q] + (in.dtvx ? in.dtvx[q] : c.dtauv) * Rx1;
      }
    }
    if (fy) {
      Fy = (in.txy[q + 1] - in.txy[q]) * c.rdx + (in.tyy[q] - in.tyy[q - px]) * c.rdy +
           (in.tyz[q + pxy] - in.tyz[q]) * c.rdz - (in.lP1[q] - in.lP1[q - px]) * c.rdy +
           in.bfy[q] * (in.mL[q - px] + in.mL[q]);
      if (in.update) {
        Ry1 = Fy * c.rrho_i + c.damp_y * Ry[q];
        Ly1 = Ly[q] + (in.dtvy ? in.dtvy[q] : c.dtauv) * Ry1;
      }
    }
    if (fz) {
      Fz = (in.txz[q + 1] - in.txz[q]) * c.rdx + (in.tyz[q + px] - in.tyz[q]) * c.rdy +
           (in.tzz[q] - in.tzz[q - pxy]) * c.rdz - (in.lP1[q] - in.lP1[q - pxy]) * c.rdz +
           in.bfz[q] * (in.mL[q - pxy] + in.mL[q]);
      if (in.update) {
        Rz1 = Fz * c.rrho_i + c.damp_z * Rz[q];
        Lz1 = Lz[q] + (in.dtvz ? in.dtvz[q] : c.dtauv) * Rz1;
      }
    }
    if (in.update) {
      if (fx) { Rx[q] = Rx1; Lx[q] = Lx1; }
      if (fy) { Ry[q] = Ry1; Ly[q] = Ly1; }
      if (fz) { Rz[q] = Rz1; Lz[q] = Lz1; }
    }
    if (fx && in.rx) in.rx[q] = Fx;
    if (fy && in.ry) in.ry[q] = Fy;
    if (fz && in.rz) in.rz[q] = Fz;
    r_v = fmax(fabs(Fx), fmax(fabs(Fy), fabs(Fz)));
  }
  if (check) block_max_atomic(r_v, red + RED_V);
}

// After a converged adjoint step: dJ/dtheta -= k (dq/dk)^T lambda_F (already in gtheta), and
// the carry g = -(dF/du_o)^T lambda into the previous step (through Pto, Pfo, Lo = log(1-phi_o)).
__global__ void __launch_bounds__(256) k_adj_carry(Box b, AdjCoef c, AdjCarry a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const long long q = cidx(b, i, j, k);
  const double lP = a.lP[q], lF = a.lF[q], lL = a.lL[q];
  a.grad[q] -= a.gtheta[q];
  a.gP[q] = c.bd_rdt * lP - c.bd_rdt_a * lF - c.beta_phi * lL;
  a.gF[q] = -c.bd_rdt_a * lP + c.bda_B_rdt * lF + c.beta_phi * lL;
  a.gphi[q] = -lL / (1.0 - a.phi_o[q]);
}

// Largest |g| of the right-hand side of an adjoint step (its convergence scale).
__global__ void __launch_bounds__(256) k_adj_gmax(Box b, const double* gP, const double* gF, const double* gphi,
                                                  unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double m = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    m = fmax(fabs(gP[q]), fmax(fabs(gF[q]), fabs(gphi[q])));
  }
  block_max_atomic(m, red + RED_GMAX);
}

// ============================================================== power-law rheology (Eq. 24)
// mu joins the unknowns with the Picard row F_mu = log mu - log mu0 + log(1 + (tau_II/tau0)^(n-1)),
// tau_II^2 = t2 = (txx^2 + tyy^2 + tzz^2)/2 + a_xy^2 + a_xz^2 + a_yz^2 (a_e: the cell's four edge
// stresses averaged), tau = m eps' with m = 2 mu/(1 + mu/Gdt) at centres and m_e from the mean of
// the edge's four centres' mu; eta = eta0 mu / phi. With f = d log(1 + x)/d t2 per cell, the
// transposed system gains (for lambda_mu the multiplier of row mu):
//   row V:   - div(S), S the pseudo-stress of lambda_mu: S_ii = m_c lambda_mu f tau_ii (centres),
//            S_e = m_e sigma_e / 2 with sigma_e = sum over the edge's four cells of lambda_mu f a_e / 2
//            (the divergence counts each shear stress in two momentum rows, so the transpose of
//            the strain rate operator is minus the divergence of the edge values halved); the
//            code keeps t - S in the adjoint stress arrays the faces kernel takes the divergence of;
//   row mu:  sum_e P_e Z_e - sum_ii Q_ii g_ii(lambda_V) + lambda_mu (1/mu + f sum tau_ii Q_ii)
//            + (Pt-Pf) cc/mu (lambda_F - lambda_P) + (Pt-Pf) dt phi/(eta0 mu^2) lambda_L - g_mu
//            with Q_ii = (dm/dmu) eps'_ii, P_e = (dm/dmu)_e eps_e / 4 over the cell's 12 edges and
//            Z_e = sigma_e - 2 eps_e(lambda_V), solved by Jacobi on its diagonal;
//   rows Pt, Pf, phi: the same as without the power law with mu per cell (cc, dt/eta, pseudo-steps).
namespace {
__device__ inline double modulus(double m, double Gdt) { return 2.0 * m / (1.0 + m / Gdt); }
__device__ inline double dmodulus(double m, double Gdt) {
  const double s = 1.0 / (1.0 + m / Gdt);
  return 2.0 * s * s;
}
}  // namespace

// Pass 1: edge moduli, P_e and the state's edge stresses (scratch), for the edges owned by the index.
__global__ void __launch_bounds__(256) k_adj_prep_pl_edges(Box b, AdjCoef c, AdjState u, AdjPrepPL pl,
                                                           double* tau_xy, double* tau_xz, double* tau_yz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  if (k < b.nz) {
    double me = 0.0, P = 0.0, t = 0.0;
    if (i > 0 && i < b.nx && j > 0 && j < b.ny) {
      const double m = 0.25 * (u.mu[q - 1 - px] + u.mu[q - px] + u.mu[q - 1] + u.mu[q]);
      const double e = 0.5 * ((u.Vx[q] - u.Vx[q - px]) * c.rdy + (u.Vy[q] - u.Vy[q - 1]) * c.rdx);
      me = modulus(m, c.Gdt);
      P = 0.25 * dmodulus(m, c.Gdt) * e;
      t = me * e;
    }
    pl.me_xy[q] = me; pl.P_xy[q] = P; tau_xy[q] = t;
  }
  if (j < b.ny) {
    double me = 0.0, P = 0.0, t = 0.0;
    if (i > 0 && i < b.nx && k > 0 && k < b.nz) {
      const double m = 0.25 * (u.mu[q - 1 - pxy] + u.mu[q - pxy] + u.mu[q - 1] + u.mu[q]);
      const double e = 0.5 * ((u.Vx[q] - u.Vx[q - pxy]) * c.rdz + (u.Vz[q] - u.Vz[q - 1]) * c.rdx);
      me = modulus(m, c.Gdt);
      P = 0.25 * dmodulus(m, c.Gdt) * e;
      t = me * e;
    }
    pl.me_xz[q] = me; pl.P_xz[q] = P; tau_xz[q] = t;
  }
  if (i < b.nx) {
    double me = 0.0, P = 0.0, t = 0.0;
    if (j > 0 && j < b.ny && k > 0 && k < b.nz) {
      const double m = 0.25 * (u.mu[q - px - pxy] + u.mu[q - pxy] + u.mu[q - px] + u.mu[q]);
      const double e = 0.5 * ((u.Vy[q] - u.Vy[q - pxy]) * c.rdz + (u.Vz[q] - u.Vz[q - px]) * c.rdy);
      me = modulus(m, c.Gdt);
      P = 0.25 * dmodulus(m, c.Gdt) * e;
      t = me * e;
    }
    pl.me_yz[q] = me; pl.P_yz[q] = P; tau_yz[q] = t;
  }
}

// Pass 2: the coefficients of k_adj_prep with mu per cell, and the power-law arrays.
__global__ void __launch_bounds__(256) k_adj_prep_pl(Box b, AdjCoef c, AdjState u, const double* __restrict__ K0,
                                                     AdjPrep o, AdjPrepPL pl, const double* __restrict__ tau_xy,
                                                     const double* __restrict__ tau_xz,
                                                     const double* __restrict__ tau_yz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  // lower faces of the cell: Darcy, advection and velocity pseudo-step coefficients
  {
    double kf = 0.0, gk = 0.0, bf = 0.0, dv = 0.0;
    if (i > 0 && i < b.nx && j < b.ny && k < b.nz) {
      const double pl_ = u.phi[q - 1], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - 1, pl_) + kperm(c, K0, q, pr)) * c.rdx * c.rdx;
      gk = -0.5 * (u.Pf[q] - u.Pf[q - 1]) * c.rdx * c.rdx;
      bf = -c.hdt_rdx * (pr - pl_);
      dv = 0.5 * c.dtauv_fac * (1.0 / u.mu[q - 1] + 1.0 / u.mu[q]);
    }
    o.kfx[q] = kf; o.gkx[q] = gk; o.bfx[q] = bf; pl.dtvx[q] = dv;
  }
  {
    double kf = 0.0, gk = 0.0, bf = 0.0, dv = 0.0;
    if (j > 0 && j < b.ny && i < b.nx && k < b.nz) {
      const double pl_ = u.phi[q - px], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - px, pl_) + kperm(c, K0, q, pr)) * c.rdy * c.rdy;
      gk = -0.5 * (u.Pf[q] - u.Pf[q - px]) * c.rdy * c.rdy;
      bf = -c.hdt_rdy * (pr - pl_);
      dv = 0.5 * c.dtauv_fac * (1.0 / u.mu[q - px] + 1.0 / u.mu[q]);
    }
    o.kfy[q] = kf; o.gky[q] = gk; o.bfy[q] = bf; pl.dtvy[q] = dv;
  }
  {
    double kf = 0.0, gk = 0.0, bf = 0.0, dv = 0.0;
    if (k > 0 && k < b.nz && i < b.nx && j < b.ny) {
      const double pl_ = u.phi[q - pxy], pr = u.phi[q];
      kf = 0.5 * (kperm(c, K0, q - pxy, pl_) + kperm(c, K0, q, pr)) * c.rdz * c.rdz;
      gk = -0.5 * ((u.Pf[q] - u.Pf[q - pxy]) * c.rdz + c.buoy) * c.rdz;
      bf = -c.hdt_rdz * (pr - pl_);
      dv = 0.5 * c.dtauv_fac * (1.0 / u.mu[q - pxy] + 1.0 / u.mu[q]);
    }
    o.kfz[q] = kf; o.gkz[q] = gk; o.bfz[q] = bf; pl.dtvz[q] = dv;
  }
  if (i >= b.nx || j >= b.ny || k >= b.nz) return;
  const double ph = u.phi[q], mu = u.mu[q], imu = 1.0 / mu;
  const double w = 1.0 / (1.0 - ph);
  const double cc = ph * w * imu * c.r_eta0;                 // 1 / (eta (1 - phi)), eta = eta0 mu / phi
  const double kc = kperm(c, K0, q, ph);
  double kmax = kc;
  if (i > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - 1, u.phi[q - 1]));
  if (i < b.nx - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + 1, u.phi[q + 1]));
  if (j > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - px, u.phi[q - px]));
  if (j < b.ny - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + px, u.phi[q + px]));
  if (k > 0) kmax = pos_max_d(kmax, kperm(c, K0, q - pxy, u.phi[q - pxy]));
  if (k < b.nz - 1) kmax = pos_max_d(kmax, kperm(c, K0, q + pxy, u.phi[q + pxy]));
  const double Pt = u.Pt[q], Pf = u.Pf[q];
  const double dt_eta = c.dt * ph * imu * c.r_eta0;           // dt / eta
  o.W[q] = w;
  o.cP[q] = 1.0 / (1.0 / (c.dtaupt_fac * mu) + c.bd_rdt + cc);
  o.cF[q] = 1.0 / (kmax * c.ifac_pf + c.bda_B_rdt + cc);
  o.aPF[q] = (Pt - Pf) * w * w * imu * c.r_eta0;
  o.a3k[q] = 3.0 * kc / ph;
  const double omc = 1.0 - ph;
  double S = 0.0, dS = 0.0;
  if (i > 0) { S += u.Vx[q] * (omc - (1.0 - u.phi[q - 1])) * c.rdx; dS -= u.Vx[q] * c.rdx; }
  if (i < b.nx - 1) { S += u.Vx[q + 1] * ((1.0 - u.phi[q + 1]) - omc) * c.rdx; dS += u.Vx[q + 1] * c.rdx; }
  if (j > 0) { S += u.Vy[q] * (omc - (1.0 - u.phi[q - px])) * c.rdy; dS -= u.Vy[q] * c.rdy; }
  if (j < b.ny - 1) { S += u.Vy[q + px] * ((1.0 - u.phi[q + px]) - omc) * c.rdy; dS += u.Vy[q + px] * c.rdy; }
  if (k > 0) { S += u.Vz[q] * (omc - (1.0 - u.phi[q - pxy])) * c.rdz; dS -= u.Vz[q] * c.rdz; }
  if (k < b.nz - 1) { S += u.Vz[q + pxy] * ((1.0 - u.phi[q + pxy]) - omc) * c.rdz; dS += u.Vz[q + pxy] * c.rdz; }
  const double diag = -w + c.dt * c.r_eta0 * imu * (Pf - Pt) + c.dt * 0.5 * (w * w * S + w * dS);
  o.Dg[q] = diag;
  o.iD[q] = 1.0 / diag;
  o.mL[q] = o.lL[q] * w;
  // ---- power law
  const double gx = (u.Vx[q + 1] - u.Vx[q]) * c.rdx, gy = (u.Vy[q + px] - u.Vy[q]) * c.rdy;
  const double gz = (u.Vz[q + pxy] - u.Vz[q]) * c.rdz;
  const double d3 = (gx + gy + gz) * c.third;
  const double exx = gx - d3, eyy = gy - d3, ezz = gz - d3;
  const double mc = modulus(mu, c.Gdt), dm = dmodulus(mu, c.Gdt);
  const double txx = mc * exx, tyy = mc * eyy, tzz = mc * ezz;
  const double axy = 0.25 * (tau_xy[q] + tau_xy[q + 1] + tau_xy[q + px] + tau_xy[q + 1 + px]);
  const double axz = 0.25 * (tau_xz[q] + tau_xz[q + 1] + tau_xz[q + pxy] + tau_xz[q + 1 + pxy]);
  const double ayz = 0.25 * (tau_yz[q] + tau_yz[q + px] + tau_yz[q + pxy] + tau_yz[q + px + pxy]);
  const double t2 = 0.5 * (txx * txx + tyy * tyy + tzz * tzz) + axy * axy + axz * axz + ayz * ayz;
  double f;                                                   // d log(1 + x) / d t2, x = (t2/tau0^2)^pw
  if (c.pw == 1.0) {
    f = c.rtau0_2 / (1.0 + t2 * c.rtau0_2);
  } else {
    const double x = t2 > 0.0 ? pow(t2 * c.rtau0_2, c.pw) : 0.0;
    f = t2 > 0.0 ? c.pw * x / ((1.0 + x) * t2) : 0.0;
  }
  const double Qxx = dm * exx, Qyy = dm * eyy, Qzz = dm * ezz;
  const double fTQ = f * (txx * Qxx + tyy * Qyy + tzz * Qzz);
  const double Axy = 0.5 * f * axy, Axz = 0.5 * f * axz, Ayz = 0.5 * f * ayz;
  pl.mc[q] = mc; pl.cc[q] = cc; pl.cplL[q] = c.beta_phi + dt_eta; pl.imu[q] = imu;
  pl.Qxx[q] = Qxx; pl.Qyy[q] = Qyy; pl.Qzz[q] = Qzz;
  pl.sTxx[q] = mc * f * txx; pl.sTyy[q] = mc * f * tyy; pl.sTzz[q] = mc * f * tzz;
  pl.Axy[q] = Axy; pl.Axz[q] = Axz; pl.Ayz[q] = Ayz;
  pl.fTQ[q] = fTQ;
  // diagonal of row mu: 1/mu + f sum tau Q + sum over the 12 edges of P_e dZ_e/dlambda_mu (= A)
  const double sP = Axy * (pl.P_xy[q] + pl.P_xy[q + 1] + pl.P_xy[q + px] + pl.P_xy[q + 1 + px]) +
                    Axz * (pl.P_xz[q] + pl.P_xz[q + 1] + pl.P_xz[q + pxy] + pl.P_xz[q + 1 + pxy]) +
                    Ayz * (pl.P_yz[q] + pl.P_yz[q + px] + pl.P_yz[q + pxy] + pl.P_yz[q + px + pxy]);
  pl.iDmu[q] = 1.0 / (imu + fTQ + sP);
  pl.cmu[q] = (Pt - Pf) * cc * imu;
  pl.cmuL[q] = (Pt - Pf) * dt_eta * imu;
}

// Edges of one iteration: sigma_e from lambda_mu, adjoint edge stress m_e (eps_e(lambda_V) - sigma_e/2),
// Z_e = sigma_e - 2 eps_e(lambda_V); zero on wall edges.
__global__ void __launch_bounds__(256) k_adj_edges_pl(Box b, AdjCoef c, AdjEdgeIn in, AdjEdgeOut out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i > b.nx || j > b.ny || k > b.nz) return;
  const long long q = cidx(b, i, j, k);
  const long long px = b.px, pxy = b.pxy;
  if (k < b.nz) {
    double t = 0.0, Z = 0.0;
    if (i > 0 && i < b.nx && j > 0 && j < b.ny) {
      const double e = 0.5 * ((in.Lx[q] - in.Lx[q - px]) * c.rdy + (in.Ly[q] - in.Ly[q - 1]) * c.rdx);
      const double sg = in.Axy[q - 1 - px] * in.lM[q - 1 - px] + in.Axy[q - px] * in.lM[q - px] +
                        in.Axy[q - 1] * in.lM[q - 1] + in.Axy[q] * in.lM[q];
      t = in.me_xy[q] * (e - 0.5 * sg);
      Z = sg - 2.0 * e;
    }
    out.txy[q] = t; out.Zxy[q] = Z;
  }
  if (j < b.ny) {
    double t = 0.0, Z = 0.0;
    if (i > 0 && i < b.nx && k > 0 && k < b.nz) {
      const double e = 0.5 * ((in.Lx[q] - in.Lx[q - pxy]) * c.rdz + (in.Lz[q] - in.Lz[q - 1]) * c.rdx);
      const double sg = in.Axz[q - 1 - pxy] * in.lM[q - 1 - pxy] + in.Axz[q - pxy] * in.lM[q - pxy] +
                        in.Axz[q - 1] * in.lM[q - 1] + in.Axz[q] * in.lM[q];
      t = in.me_xz[q] * (e - 0.5 * sg);
      Z = sg - 2.0 * e;
    }
    out.txz[q] = t; out.Zxz[q] = Z;
  }
  if (i < b.nx) {
    double t = 0.0, Z = 0.0;
    if (j > 0 && j < b.ny && k > 0 && k < b.nz) {
      const double e = 0.5 * ((in.Ly[q] - in.Ly[q - pxy]) * c.rdz + (in.Lz[q] - in.Lz[q - px]) * c.rdy);
      const double sg = in.Ayz[q - px - pxy] * in.lM[q - px - pxy] + in.Ayz[q - pxy] * in.lM[q - pxy] +
                        in.Ayz[q - px] * in.lM[q - px] + in.Ayz[q] * in.lM[q];
      t = in.me_yz[q] * (e - 0.5 * sg);
      Z = sg - 2.0 * e;
    }
    out.tyz[q] = t; out.Zyz[q] = Z;
  }
}

// Cells (power law): centre adjoint stresses minus the pseudo-stress, rows Pt, Pf, phi with mu per
// cell, and row mu.
__global__ void __launch_bounds__(256) k_adj_cells_pl(Box b, AdjCoef c, AdjState u, AdjCellIn in, AdjCellOut out,
                                                      AdjPrepPL pl, AdjMuIn mi, unsigned long long* red,
                                                      int check) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double r_pt = 0.0, r_pf = 0.0, r_l = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    const double ph = u.phi[q];
    const double cc = pl.cc[q];
    const double lP = in.lP[q], lF = in.lF[q], lL = in.lL[q], lM = mi.lM[q];
    const double Lz0 = in.Lz[q], Lz1 = in.Lz[q + pxy];
    const double gx = (in.Lx[q + 1] - in.Lx[q]) * c.rdx, gy = (in.Ly[q + px] - in.Ly[q]) * c.rdy;
    const double gz = (Lz1 - Lz0) * c.rdz;
    const double divL = gx + gy + gz;
    const double d3 = divL * c.third;
    const double mc = pl.mc[q];
    out.txx[q] = mc * (gx - d3) - lM * pl.sTxx[q];
    out.tyy[q] = mc * (gy - d3) - lM * pl.sTyy[q];
    out.tzz[q] = mc * (gz - d3) - lM * pl.sTzz[q];
    // ---- row Pt
    const double cplP = c.bd_rdt_a + cc, cplL = pl.cplL[q];
    const double resP = divL + (c.bd_rdt + cc) * lP - cplP * lF - cplL * lL - in.gP[q];
    out.lP[q] = lP - in.cP[q] * resP;
    // ---- row Pf and the advection transpose of row phi over the six faces
    double Klf = 0.0, dkT = 0.0, offx = 0.0, offy = 0.0, offz = 0.0;
    if (i > 0) {
      const double dn = in.lF[q - 1] - lF;
      Klf -= in.kfx[q] * dn;
      dkT += in.gkx[q] * dn;
      offx -= u.Vx[q] * in.mL[q - 1];
    }
    if (i < b.nx - 1) {
      const double dn = in.lF[q + 1] - lF;
      Klf -= in.kfx[q + 1] * dn;
      dkT -= in.gkx[q + 1] * dn;
      offx += u.Vx[q + 1] * in.mL[q + 1];
    }
    if (j > 0) {
      const double dn = in.lF[q - px] - lF;
      Klf -= in.kfy[q] * dn;
      dkT += in.gky[q] * dn;
      offy -= u.Vy[q] * in.mL[q - px];
    }
    if (j < b.ny - 1) {
      const double dn = in.lF[q + px] - lF;
      Klf -= in.kfy[q + px] * dn;
      dkT -= in.gky[q + px] * dn;
      offy += u.Vy[q + px] * in.mL[q + px];
    }
    if (k > 0) {
      const double dn = in.lF[q - pxy] - lF;
      Klf -= in.kfz[q] * dn;
      dkT += in.gkz[q] * dn;
      offz -= u.Vz[q] * in.mL[q - pxy];
    }
    if (k < b.nz - 1) {
      const double dn = in.lF[q + pxy] - lF;
      Klf -= in.kfz[q + pxy] * dn;
      dkT -= in.gkz[q + pxy] * dn;
      offz += u.Vz[q + pxy] * in.mL[q + pxy];
    }
    const double off = offx * c.hdt_rdx + offy * c.hdt_rdy + offz * c.hdt_rdz;
    const double resF = Klf + (c.bda_B_rdt + cc) * lF - cplP * lP + cplL * lL - in.gF[q];
    out.lF[q] = lF - in.cF[q] * resF;
    const double a3k = in.a3k[q];
    if (out.gtheta) out.gtheta[q] = a3k * ph * c.third * dkT;
    // ---- row phi
    const double sL = -c.hdrho_g * (Lz0 + Lz1) + in.aPF[q] * (lP - lF) + a3k * dkT + off - in.gphi[q];
    const double lLn = -in.iD[q] * sL;
    out.lL[q] = lLn;
    out.mL[q] = lLn * in.W[q];
    // ---- row mu
    const double sPZ =
        pl.P_xy[q] * mi.Zxy[q] + pl.P_xy[q + 1] * mi.Zxy[q + 1] + pl.P_xy[q + px] * mi.Zxy[q + px] +
        pl.P_xy[q + 1 + px] * mi.Zxy[q + 1 + px] + pl.P_xz[q] * mi.Zxz[q] + pl.P_xz[q + 1] * mi.Zxz[q + 1] +
        pl.P_xz[q + pxy] * mi.Zxz[q + pxy] + pl.P_xz[q + 1 + pxy] * mi.Zxz[q + 1 + pxy] +
        pl.P_yz[q] * mi.Zyz[q] + pl.P_yz[q + px] * mi.Zyz[q + px] + pl.P_yz[q + pxy] * mi.Zyz[q + pxy] +
        pl.P_yz[q + px + pxy] * mi.Zyz[q + px + pxy];
    const double resM = sPZ - (pl.Qxx[q] * gx + pl.Qyy[q] * gy + pl.Qzz[q] * gz) +
                        lM * (pl.imu[q] + pl.fTQ[q]) + pl.cmu[q] * (lF - lP) + pl.cmuL[q] * lL - mi.gM[q];
    mi.lM1[q] = lM - pl.iDmu[q] * resM;
    if (check || out.rL) {
      const double resL = sL + in.Dg[q] * lL;
      if (out.rL) {
        out.rP[q] = resP;
        out.rF[q] = resF;
        out.rL[q] = resL;
      }
      if (mi.rM) mi.rM[q] = resM;
      r_pt = fabs(resP);
      r_pf = fabs(resF);
      r_l = fmax(fabs(resL), fabs(resM));
      if (!(resL == resL && resM == resM)) r_l = resL + resM;   // a NaN surfaces in the norm
    }
  }
  if (check) {
    block_max_atomic(r_pt, red + RED_PT);
    block_max_atomic(r_pf, red + RED_PF);
    block_max_atomic(r_l, red + RED_PIC);
  }
}

// d(lambda . F)/d(G dtS): the moduli depend on Gdt through xi = mu / Gdt; summed over the grid.
__global__ void __launch_bounds__(256) k_adj_dgdt_pl(Box b, AdjCoef c, AdjState u, AdjPrepPL pl,
                                                     const double* __restrict__ Lx, const double* __restrict__ Ly,
                                                     const double* __restrict__ Lz, const double* __restrict__ lM,
                                                     const double* __restrict__ Zxy, const double* __restrict__ Zxz,
                                                     const double* __restrict__ Zyz, double* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double v = 0.0;
  if (i <= b.nx && j <= b.ny && k <= b.nz) {
    const long long q = cidx(b, i, j, k);
    const long long px = b.px, pxy = b.pxy;
    if (i < b.nx && j < b.ny && k < b.nz) {
      const double r = u.mu[q] / c.Gdt;
      const double gx = (Lx[q + 1] - Lx[q]) * c.rdx, gy = (Ly[q + px] - Ly[q]) * c.rdy;
      const double gz = (Lz[q + pxy] - Lz[q]) * c.rdz;
      v += r * r * (-(pl.Qxx[q] * gx + pl.Qyy[q] * gy + pl.Qzz[q] * gz) + lM[q] * pl.fTQ[q]);
    }
    if (k < b.nz && i > 0 && i < b.nx && j > 0 && j < b.ny) {
      const double r = 0.25 * (u.mu[q - 1 - px] + u.mu[q - px] + u.mu[q - 1] + u.mu[q]) / c.Gdt;
      v += 4.0 * pl.P_xy[q] * r * r * Zxy[q];
    }
    if (j < b.ny && i > 0 && i < b.nx && k > 0 && k < b.nz) {
      const double r = 0.25 * (u.mu[q - 1 - pxy] + u.mu[q - pxy] + u.mu[q - 1] + u.mu[q]) / c.Gdt;
      v += 4.0 * pl.P_xz[q] * r * r * Zxz[q];
    }
    if (i < b.nx && j > 0 && j < b.ny && k > 0 && k < b.nz) {
      const double r = 0.25 * (u.mu[q - px - pxy] + u.mu[q - pxy] + u.mu[q - px] + u.mu[q]) / c.Gdt;
      v += 4.0 * pl.P_yz[q] * r * r * Zyz[q];
    }
  }
  // block sum, then one atomic add per block
  __shared__ double part[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int t = threadIdx.x + blockDim.x * threadIdx.y, lane = t & 31, warp = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) part[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? part[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0 && v != 0.0) atomicAdd(acc, v);
  }
}

__global__ void __launch_bounds__(256) k_adj_mumax(Box b, const double* __restrict__ mu, unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  double m = 0.0;
  if (i < b.nx && j < b.ny && k < b.nz) m = mu[cidx(b, i, j, k)];
  block_max_atomic(m, red + RED_MUMAX);
}
__global__ void __launch_bounds__(256) k_adj_argmax(Box b, const double* __restrict__ mu, unsigned long long* red) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i < b.nx && j < b.ny && k < b.nz) {
    const long long q = cidx(b, i, j, k);
    if ((unsigned long long)__double_as_longlong(mu[q]) == red[RED_MUMAX]) atomicMin(red + RED_ARG, (unsigned long long)q);
  }
}
__global__ void k_adj_add_at(double* gM, long long n, const unsigned long long* red, const double* acc,
                             double scale) {
  const unsigned long long q = red[RED_ARG];
  if (threadIdx.x == 0 && blockIdx.x == 0 && q < (unsigned long long)n) gM[q] += scale * (*acc);
}

void adj_prep_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const double* K0,
                 const AdjPrep& out, const AdjPrepPL& pl, double* tau_xy, double* tau_xz, double* tau_yz) {
  k_adj_prep_pl_edges<<<g, bl, 0, s>>>(b, c, u, pl, tau_xy, tau_xz, tau_yz);
  k_adj_prep_pl<<<g, bl, 0, s>>>(b, c, u, K0, out, pl, tau_xy, tau_xz, tau_yz);
}
void adj_edges_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjEdgeIn& in,
                  const AdjEdgeOut& out) {
  k_adj_edges_pl<<<g, bl, 0, s>>>(b, c, in, out);
}
void adj_cells_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
                  const AdjCellOut& out, const AdjPrepPL& pl, const AdjMuIn& mu, unsigned long long* red,
                  int check) {
  k_adj_cells_pl<<<g, bl, 0, s>>>(b, c, u, in, out, pl, mu, red, check);
}
void adj_dgdt_pl(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u,
                 const AdjPrepPL& pl, const double* Lx, const double* Ly, const double* Lz, const double* lM,
                 const double* Zxy, const double* Zxz, const double* Zyz, double* acc) {
  k_adj_dgdt_pl<<<g, bl, 0, s>>>(b, c, u, pl, Lx, Ly, Lz, lM, Zxy, Zxz, Zyz, acc);
}
void adj_argmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* mu, unsigned long long* red) {
  k_adj_mumax<<<g, bl, 0, s>>>(b, mu, red);
  k_adj_argmax<<<g, bl, 0, s>>>(b, mu, red);
}
void adj_add_at(cudaStream_t s, Box b, double* gM, const unsigned long long* red, const double* acc,
                double scale) {
  k_adj_add_at<<<1, 32, 0, s>>>(gM, b.n, red, acc, scale);
}

void adj_prep(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const double* K0,
              const AdjPrep& out) {
  k_adj_prep<<<g, bl, 0, s>>>(b, c, u, K0, out);
}
void adj_cells(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjState& u, const AdjCellIn& in,
               const AdjCellOut& out, unsigned long long* red, int check) {
  k_adj_cells<<<g, bl, 0, s>>>(b, c, u, in, out, red, check);
}
void adj_faces(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjFaceIn& in, double* Lx,
               double* Ly, double* Lz, double* Rx, double* Ry, double* Rz, unsigned long long* red, int check) {
  k_adj_faces<<<g, bl, 0, s>>>(b, c, in, Lx, Ly, Lz, Rx, Ry, Rz, red, check);
}
void adj_carry(dim3 g, dim3 bl, cudaStream_t s, Box b, const AdjCoef& c, const AdjCarry& a) {
  k_adj_carry<<<g, bl, 0, s>>>(b, c, a);
}
void adj_gmax(dim3 g, dim3 bl, cudaStream_t s, Box b, const double* gP, const double* gF, const double* gphi,
              unsigned long long* red) {
  k_adj_gmax<<<g, bl, 0, s>>>(b, gP, gF, gphi, red);
}

}  // namespace pt
